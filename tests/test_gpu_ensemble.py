"""Adjoint statistics of Sec. IV (da_adjoint_spectra): shell energies of the
adjoint velocity per member and of the ensemble-mean adjoint, at every saved
backward time, against the oracle's adjoint states."""
import numpy as np
import pytest

from cases import make_pair
from paper_2602_14016_gb300 import synthetic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a GPU")
    from paper_2602_14016_gb300 import api as A, build

    build.build()
    return A


def shell_energy(lam_hat, n):
    """E(k) = 1/2 sum_{k <= |k| < k+1} |u_dagger_hat|^2, u_dagger = (dy lam, -dx lam),
    normalised coefficients, from a half spectrum (kx > 0 stands for +-kx)."""
    KX, KY = synthetic.wavenumbers(n)
    k2 = (KX**2 + KY**2).astype(float)
    mask = synthetic.retained_mask(n) & (k2 > 0)
    K = (n - 1) // 3
    nshell = int(np.floor(np.sqrt(2.0) * K)) + 1
    wgt = np.where(KX == 0, 1.0, 2.0) * k2 / (2.0 * n**4)
    sh = np.floor(np.sqrt(k2)).astype(int)
    e = np.zeros(nshell)
    np.add.at(e, sh[mask], (wgt * np.abs(lam_hat) ** 2)[mask])
    return e


def oracle_adjoint_states(orc, P, s, lamT):
    """lambda_k for k = nsteps..0, by the oracle's step transposes."""
    _, _, traj = orc.forward(P, s, trajectory=True)
    lam = np.where(synthetic.retained_mask(P.n), lamT, 0)
    out = {P.nsteps: lam}
    for k in range(P.nsteps - 1, -1, -1):
        lam = orc.step_adj(P, traj[k], lam)
        out[k] = lam
    return out


@pytest.mark.parametrize("ckpt", [0, 5])
def test_adjoint_spectra_against_oracle(orc, api, ckpt):
    n, nsteps, every, B = 32, 12, 4, 3
    probs, cfg = make_pair(orc, n, nsteps, 5e-3, 5e-4, kernels=[("identity", 0.0)] * B, px=8, every=4)
    cfg.ckpt_every = ckpt
    ctx = api.Context(cfg)
    ws = [synthetic.random_vorticity_hat(n, 200 + b) * 2 for b in range(B)]
    s = np.stack([orc.control_from_omega(probs[b], ws[b]) for b in range(B)])
    lamT = np.stack([synthetic.unit_norm_terminal_hat(n, 300 + b) for b in range(B)])
    member, mean = ctx.adjoint_spectra(torch.from_numpy(s).cuda(), torch.from_numpy(lamT).cuda(), every)
    member, mean = member.cpu().numpy(), mean.cpu().numpy()
    states = [oracle_adjoint_states(orc, probs[b], s[b], lamT[b]) for b in range(B)]
    for slot, k in enumerate(range(nsteps, -1, -every)):
        for b in range(B):
            ref = shell_energy(states[b][k], n)
            assert np.abs(member[b, slot] - ref).max() <= 1e-10 * ref.max()
        ref_mean = shell_energy(sum(states[b][k] for b in range(B)) / B, n)
        assert np.abs(mean[slot] - ref_mean).max() <= 1e-10 * ref_mean.max()
    # energy identity at tau = 0: sum_k E(k) = 1/2 mean over the grid of |u_dagger|^2
    KX, KY = synthetic.wavenumbers(n)
    lam = np.where(synthetic.retained_mask(n), lamT[0], 0)
    ux = np.fft.irfft2(1j * KY * lam, s=(n, n))
    uy = np.fft.irfft2(-1j * KX * lam, s=(n, n))
    assert abs(member[0, 0].sum() - 0.5 * np.mean(ux**2 + uy**2)) < 1e-12 * member[0, 0].sum()


@pytest.mark.parametrize("ckpt", [0, 4])
def test_graph_replayed_spectra_equal_direct_launches(api, ckpt):
    """da_adjoint_spectra under da_set_graphs: the captured sequence, replayed
    twice (the second time on new inputs), gives bitwise the direct launches'
    spectra and gradient state."""
    n, B, nsteps = 32, 3, 12
    cfg = api.Config(n=n, nsteps=nsteps, dt=5e-3, nu=1e-3, px=1, every=nsteps, ckpt_every=ckpt,
                     kernels=[api.KernelSpec("identity", 0.0)] * B)
    direct, graph = api.Context(cfg), api.Context(cfg)
    graph.set_graphs(True)
    for rep in range(2):
        w = torch.from_numpy(np.stack([synthetic.random_vorticity_hat(n, 50 * rep + b) for b in range(B)])).cuda()
        s = direct.control_from_omega(w)
        lamT = torch.from_numpy(np.stack([synthetic.unit_norm_terminal_hat(n, 90 + 50 * rep + b)
                                          for b in range(B)])).cuda()
        m1, e1 = direct.adjoint_spectra(s, lamT, 3)
        m2, e2 = graph.adjoint_spectra(s, lamT, 3)
        l1, _ = direct.last_adjoint()
        l2, _ = graph.last_adjoint()
        torch.cuda.synchronize()
        assert torch.equal(m1, m2) and torch.equal(e1, e2) and torch.equal(l1, l2)
