// blas.cuh -- per-member vector kernels of the optimiser (L-BFGS, Sec. II.C).
//
// Every member of a batch owns a set of vectors of `len` doubles in one bank
// buffer: bank k of member b starts at V + (k * B + b) * len.  Banks:
// x, g, d (search direction), xt, gt (trial point and its gradient), then
// the S slots and the Y slots of the pair ring.  One CTA serves one member
// (blockIdx.x = member), so every reduction is a CTA tree reduction in a
// fixed order: results are bitwise reproducible, and the two-loop recursion
// runs as one launch with all of its scalars on the device.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace da {

enum : int { BANK_X = 0, BANK_G = 1, BANK_D = 2, BANK_XT = 3, BANK_GT = 4, BANK_S0 = 5 };

// Device scalars per member, [B][SC_COUNT].
enum : int { SC_J = 0, SC_GG = 1, SC_GD = 2, SC_DG = 3, SC_SY = 4, SC_YY = 5, SC_COUNT = 6 };

constexpr int kBlasThreads = 512;

// Per-call arguments uploaded by the host (one small copy per phase).
struct LbfgsArgs {
  double* V;            // banks
  size_t len;           // doubles per vector
  int B, slots;         // members; S slots at BANK_S0 + t, Y slots at BANK_S0 + slots + t
  int mem;              // pair capacity (slots - 1)
  double* scal;         // [B][SC_COUNT]
  const int* mask;      // [B] member takes part in this launch
  const int* cnt;       // [B] pairs held (two-loop)
  const int* pslot;     // [B][mem] slot of each pair, oldest first
  const double* prho;   // [B][mem] 1 / (s . y) of each pair
  const double* stp;    // [B] trial step
  const int* aslot;     // [B] slot that receives an accepted pair
};

// d = -H g by the two-loop recursion with H0 = (s.y / y.y) I from the
// newest pair, then scal[GD] = g . d.  grid B, block kBlasThreads.
__global__ void k_two_loop(LbfgsArgs a);
// d = -g for masked members.  grid (chunks, B).
__global__ void k_neg_grad(LbfgsArgs a);
// xt = x + stp d for masked members, xt = x for the others.  grid (chunks, B).
__global__ void k_trial(LbfgsArgs a);
// scal[DG] = gt . d for masked members.  grid B.
__global__ void k_dot_gt_d(LbfgsArgs a);
// Masked members accept their trial: S[aslot] = xt - x, Y[aslot] = gt - g,
// scal[SY], scal[YY], x = xt, g = gt.  grid B.
__global__ void k_accept(LbfgsArgs a);
// scal[GG] = g . g for every member.  grid B.
__global__ void k_gnorm2(LbfgsArgs a);
// g = gt for masked members (their first evaluation).  grid (chunks, B).
__global__ void k_take_gradient(LbfgsArgs a);

}  // namespace da
