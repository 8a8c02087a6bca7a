// linesearch.h -- strong-Wolfe line search of More and Thuente (ACM TOMS 20,
// 1994) as a resumable state machine, so that the members of a batch can
// search together: each call of step() consumes phi(stp) and phi'(stp) of the
// last trial and says whether to evaluate a new trial step.
//
// The search keeps an interval of uncertainty [stx, sty] and proposes trials
// from cubic and quadratic (secant) interpolants of the end points, with the
// safeguards of the paper: extrapolation is bounded by [1.1, 4] times the
// last step until a minimiser is bracketed, the interval must shrink by a
// factor 0.66 every two trials or the trial bisects it, and while the
// sufficient-decrease function psi(a) = phi(a) - c1 a phi'(0) has not gone
// non-positive with non-negative slope, the interval is updated on psi.
#pragma once
#include <algorithm>
#include <cmath>

namespace da {

class MoreThuente {
 public:
  enum Action { EVALUATE = 0, CONVERGED = 1, FAILED = 2 };

  void start(double f0, double g0, double stp0, double c1, double c2, double xtol, double stpmin, double stpmax,
             int max_evals) {
    f0_ = f0;
    g0_ = g0;
    c1_ = c1;
    c2_ = c2;
    xtol_ = xtol;
    smin_ = stpmin;
    smax_ = stpmax;
    max_evals_ = max_evals;
    evals_ = 0;
    bracketed_ = false;
    aux_ = true;
    width_ = smax_ - smin_;
    width_prev_ = 2.0 * width_;
    lx_ = 0.0; fx_ = f0; dx_ = g0;
    ly_ = 0.0; fy_ = f0; dy_ = g0;
    stp_ = stp0;
    lo_ = 0.0;
    hi_ = stp0 + 4.0 * stp0;
    bad_start_ = !(g0 < 0.0) || !(stp0 > 0.0);
  }

  double stp() const { return stp_; }
  int evals() const { return evals_; }

  // phi(stp) = f, phi'(stp) = g of the trial just evaluated.
  int step(double f, double g) {
    if (bad_start_) return FAILED;
    ++evals_;
    const double slope = c1_ * g0_;
    const double armijo = f0_ + stp_ * slope;
    if (aux_ && f <= armijo && g >= 0.0) aux_ = false;
    if (f <= armijo && std::fabs(g) <= c2_ * (-g0_)) return CONVERGED;
    if (bracketed_ && (stp_ <= lo_ || stp_ >= hi_)) return FAILED;
    if (bracketed_ && hi_ - lo_ <= xtol_ * hi_) return FAILED;
    if (stp_ == smax_ && f <= armijo && g <= slope) return FAILED;
    if (stp_ == smin_ && (f > armijo || g >= slope)) return FAILED;
    if (evals_ >= max_evals_) return FAILED;

    double next;
    if (aux_ && f <= fx_ && f > armijo) {
      // update the interval on psi = phi - slope * a
      double fx = fx_ - lx_ * slope, dx = dx_ - slope;
      double fy = fy_ - ly_ * slope, dy = dy_ - slope;
      next = update(fx, dx, fy, dy, f - stp_ * slope, g - slope);
      fx_ = fx + lx_ * slope;
      dx_ = dx + slope;
      fy_ = fy + ly_ * slope;
      dy_ = dy + slope;
    } else {
      next = update(fx_, dx_, fy_, dy_, f, g);
    }
    if (bracketed_) {
      if (std::fabs(ly_ - lx_) >= 0.66 * width_prev_) next = lx_ + 0.5 * (ly_ - lx_);
      width_prev_ = width_;
      width_ = std::fabs(ly_ - lx_);
      lo_ = std::min(lx_, ly_);
      hi_ = std::max(lx_, ly_);
    } else {
      lo_ = next + 1.1 * (next - lx_);
      hi_ = next + 4.0 * (next - lx_);
    }
    next = std::min(std::max(next, smin_), smax_);
    if (bracketed_ && (next <= lo_ || next >= hi_ || hi_ - lo_ <= xtol_ * hi_)) next = lx_;
    stp_ = next;
    return EVALUATE;
  }

 private:
  // Minimiser of the cubic through (a, fa, da) and (b, fb, db).
  static double cubic(double a, double fa, double da, double b, double fb, double db) {
    const double th = 3.0 * (fa - fb) / (b - a) + da + db;
    const double sc = std::max(std::fabs(th), std::max(std::fabs(da), std::fabs(db)));
    double gm = sc * std::sqrt(std::max(0.0, (th / sc) * (th / sc) - (da / sc) * (db / sc)));
    if (b < a) gm = -gm;
    const double p = (gm - da) + th;
    const double q = ((gm - da) + gm) + db;
    return a + (p / q) * (b - a);
  }

  // One interval update with the trial (stp_, ft, gt); end points carried in
  // (lx_, fx, dx), (ly_, fy, dy).  Returns the next trial step.
  double update(double& fx, double& dx, double& fy, double& dy, double ft, double gt) {
    const double t = stp_;
    const bool sign_change = gt * (dx < 0.0 ? -1.0 : 1.0) < 0.0;
    double next;
    if (ft > fx) {
      const double c = cubic(lx_, fx, dx, t, ft, gt);
      const double qd = lx_ + (dx / ((fx - ft) / (t - lx_) + dx)) / 2.0 * (t - lx_);
      next = std::fabs(c - lx_) < std::fabs(qd - lx_) ? c : c + (qd - c) / 2.0;
      bracketed_ = true;
    } else if (sign_change) {
      const double c = cubic(t, ft, gt, lx_, fx, dx);
      const double sec = t + (gt / (gt - dx)) * (lx_ - t);
      next = std::fabs(c - t) > std::fabs(sec - t) ? c : sec;
      bracketed_ = true;
    } else if (std::fabs(gt) < std::fabs(dx)) {
      const double th = 3.0 * (fx - ft) / (t - lx_) + dx + gt;
      const double sc = std::max(std::fabs(th), std::max(std::fabs(dx), std::fabs(gt)));
      double gm = sc * std::sqrt(std::max(0.0, (th / sc) * (th / sc) - (dx / sc) * (gt / sc)));
      if (t > lx_) gm = -gm;
      const double p = (gm - gt) + th;
      const double q = (gm + (dx - gt)) + gm;
      const double rr = p / q;
      double c;
      if (rr < 0.0 && gm != 0.0)
        c = t + rr * (lx_ - t);
      else
        c = t > lx_ ? hi_ : lo_;
      const double sec = t + (gt / (gt - dx)) * (lx_ - t);
      if (bracketed_) {
        next = std::fabs(c - t) < std::fabs(sec - t) ? c : sec;
        const double lim = t + 0.66 * (ly_ - t);
        next = t > lx_ ? std::min(lim, next) : std::max(lim, next);
      } else {
        next = std::fabs(c - t) > std::fabs(sec - t) ? c : sec;
        next = std::min(hi_, std::max(lo_, next));
      }
    } else {
      if (bracketed_)
        next = cubic(t, ft, gt, ly_, fy, dy);
      else
        next = t > lx_ ? hi_ : lo_;
    }
    if (ft > fx) {
      ly_ = t;
      fy = ft;
      dy = gt;
    } else {
      if (sign_change) {
        ly_ = lx_;
        fy = fx;
        dy = dx;
      }
      lx_ = t;
      fx = ft;
      dx = gt;
    }
    return next;
  }

  double f0_ = 0, g0_ = 0, c1_ = 1e-4, c2_ = 0.9, xtol_ = 1e-10, smin_ = 0, smax_ = 1e20;
  double lx_ = 0, fx_ = 0, dx_ = 0, ly_ = 0, fy_ = 0, dy_ = 0;
  double stp_ = 1, lo_ = 0, hi_ = 0, width_ = 0, width_prev_ = 0;
  int evals_ = 0, max_evals_ = 20;
  bool bracketed_ = false, aux_ = true, bad_start_ = false;
};

}  // namespace da
