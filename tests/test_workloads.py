"""Host-side helpers of the workloads (no GPU): the first guess from the t = 0
probe velocities (the paper's initial interpolated state, Sec. III.A) and the
initial-condition error of an assimilation (Sec. III)."""
import numpy as np

from paper_2602_14016_gb300 import synthetic, workloads


def band_limited(n, kmax, seed):
    """A random vorticity half spectrum on |kx|, |ky| < kmax (zero mean)."""
    h = synthetic.random_retained_hat(n, seed)
    KX, KY = synthetic.wavenumbers(n)
    h = np.where((np.abs(KX) < kmax) & (np.abs(KY) < kmax), h, 0)
    h[0, 0] = 0
    return h


def test_probe_interpolation_recovers_fields_resolved_by_the_probes():
    """A field whose modes all lie below the probe lattice's Nyquist
    wavenumber is recovered exactly from its velocities at the probes."""
    n, px = 64, 16
    w = band_limited(n, px // 2, 3)
    # the kx = 0 column of a real field's half spectrum is Hermitian
    col = w[:, 0].copy()
    w[:, 0] = 0.5 * (col + np.conj(col[(-np.arange(n)) % n]))
    g = workloads.first_guess_from_probes(w, n, px)
    assert np.abs(g - w).max() < 1e-12 * np.abs(w).max()


def test_probe_interpolation_drops_unresolved_scales():
    n, px = 64, 8
    w = synthetic.random_vorticity_hat(n, 5)
    g = workloads.first_guess_from_probes(w, n, px)
    KX, KY = synthetic.wavenumbers(n)
    assert np.all(g[(np.abs(KX) >= px // 2) | (np.abs(KY) >= px // 2)] == 0)


def test_initial_velocity_error():
    n = 32
    w = synthetic.random_vorticity_hat(n, 1)
    assert workloads.initial_velocity_error(w, w) == 0.0
    assert abs(workloads.initial_velocity_error(1.25 * w, w) - 0.25) < 1e-14
    assert abs(workloads.initial_velocity_error(0 * w, w) - 1.0) < 1e-14
    # the metric is the velocity's: against a grid computation of u, v
    d = synthetic.random_vorticity_hat(n, 2) * 0.1
    KX, KY = synthetic.wavenumbers(n)
    k2 = np.where(KX**2 + KY**2 > 0, KX**2 + KY**2, 1.0)

    def vel(h):
        return np.fft.irfft2(1j * KY * h / k2, s=(n, n)), np.fft.irfft2(-1j * KX * h / k2, s=(n, n))

    u0, v0 = vel(w)
    u1, v1 = vel(w + d)
    expect = np.sqrt(np.sum((u1 - u0) ** 2 + (v1 - v0) ** 2) / np.sum(u0**2 + v0**2))
    assert abs(workloads.initial_velocity_error(w + d, w) - expect) < 1e-12
