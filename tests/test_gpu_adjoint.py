"""GPU adjoint of the mechanical increments (gradient of a stress-strain misfit with respect to
k1, k2, tau0, n) against the oracle's FP64 adjoint and against central finite differences."""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1509_04953_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_04953_gb300 import build
    build.build()
    from paper_1509_04953_gb300 import evp
    return evp


N, G, T, SEED = 8, 4, 4, 7


def setup_inputs():
    g0 = O.voronoi(N, synth.voronoi_seeds(N, G, SEED))
    q = synth.orientations(G, SEED)
    return g0, q


def perturbed(mat):
    return dataclasses.replace(mat, k1=mat.k1 * 1.1, k2=mat.k2 * 0.9, tau0=mat.tau0 * 1.2, n=mat.n * 1.05)


def gpu_loss_grad(ev, mat, target, precision="fp64", ck=2, tol=1e-12, adj_tol=1e-11, want_grad=True):
    g0, q = setup_inputs()
    s = ev.Solver(N, G, g0, q, mat, SEED, precision=precision, tol=tol, max_iter=20000)
    s.adjoint_begin(T, ck)
    curve = np.array([s.adjoint_step(-1e-3, 1.0).sig_mean[2] for _ in range(T)])
    L = float(((curve - target) ** 2).sum())
    grad = None
    if want_grad:
        gb = np.zeros((T, 6))
        gb[:, 2] = 2 * (curve - target)
        grad = s.adjoint_end(gb, tol=adj_tol)
    return L, grad, curve, s


@pytest.fixture(scope="module")
def target(mat):
    g0, q = setup_inputs()
    rc, _, _, tg = O.loss_grad(N, G, g0, q, mat, SEED, T, -1e-3, 1.0, want_grad=False)
    assert rc == 0
    return tg


def test_gpu_adjoint_matches_oracle_adjoint_fp64(ev, mat, target):
    m1 = perturbed(mat)
    g0, q = setup_inputs()
    rc, Lo, go, _ = O.loss_grad(N, G, g0, q, m1, SEED, T, -1e-3, 1.0, target=target)
    L, g, _, _ = gpu_loss_grad(ev, m1, target)
    assert abs(L / Lo - 1) < 1e-9
    assert np.abs(g / go - 1).max() < 1e-6, (g, go)


def test_gpu_adjoint_matches_central_differences(ev, mat, target):
    m1 = perturbed(mat)
    L, g, _, _ = gpu_loss_grad(ev, m1, target)
    for i, k in enumerate(("k1", "k2", "tau0", "n")):
        v = getattr(m1, k)
        h = 1e-6 * v
        Lp = gpu_loss_grad(ev, dataclasses.replace(m1, **{k: v + h}), target, want_grad=False)[0]
        Lm = gpu_loss_grad(ev, dataclasses.replace(m1, **{k: v - h}), target, want_grad=False)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(g[i] / fd - 1) < 1e-5, (k, g[i], fd)


def test_checkpoint_interval_does_not_change_the_gradient(ev, mat, target):
    m1 = perturbed(mat)
    grads = [gpu_loss_grad(ev, m1, target, ck=ck)[1] for ck in (1, 3, T)]
    for gr in grads[1:]:
        assert np.array_equal(gr, grads[0])


def test_state_is_restored_after_the_reverse_sweep(ev, mat, target):
    m1 = perturbed(mat)
    g0, q = setup_inputs()
    s = ev.Solver(N, G, g0, q, m1, SEED, precision="fp64", tol=1e-12, max_iter=20000)
    s.adjoint_begin(T, 2)
    for _ in range(T):
        s.adjoint_step(-1e-3, 1.0)
    before = {f: s.get(f) for f in ("sig", "epsp", "rho", "epse", "deps")}
    sc = s.scalars()
    s.adjoint_end(np.ones((T, 6)))
    for f, v in before.items():
        assert np.array_equal(s.get(f), v), f
    assert np.array_equal(s.scalars()["E"], sc["E"])
    rc, st = s.increment(-1e-3, 1.0)       # the run continues from the recorded end state
    assert rc == 0


def test_mixed_adjoint_close_to_fp64(ev, mat, target):
    m1 = perturbed(mat)
    _, g64, _, _ = gpu_loss_grad(ev, m1, target)
    # the adjoint fixed point solved to 1e-6 (FP32 fields reach it); at 1e-5 the gradient is within 1.1e-4
    _, g32, _, _ = gpu_loss_grad(ev, m1, target, precision="mixed", tol=1e-6, adj_tol=1e-6)
    assert np.abs(g32 / g64 - 1).max() < 3e-5, (g32, g64)      # measured 1.0e-5 (the n component)


def test_mixed_adjoint_against_central_differences(ev, mat, target):
    """The FP32-mixed adjoint against central differences. (1) Of the FP64 forward at h = 1e-6 relative, the
    difference quotient is accurate to about 1e-8, so the comparison measures the mixed adjoint itself: within
    3e-5 (measured 1.0e-5). (2) Of the mixed forward: its loss carries FP32 rounding and the 1e-6 fixed-point
    tolerance, about 1e-7 relative, so a quotient at h = 1e-6 is noise (the +h and -h losses can round to the
    same value) and at h <= 1e-4 it is off by percents; h = 1e-2 balances noise against truncation and agrees to
    1e-3 (measured 4.4e-4, on k2, the smallest component)."""
    m1 = perturbed(mat)
    _, g32, _, _ = gpu_loss_grad(ev, m1, target, precision="mixed", tol=1e-6, adj_tol=1e-6)
    for i, k in enumerate(("k1", "k2", "tau0", "n")):
        v = getattr(m1, k)
        h = 1e-6 * v
        Lp = gpu_loss_grad(ev, dataclasses.replace(m1, **{k: v + h}), target, want_grad=False)[0]
        Lm = gpu_loss_grad(ev, dataclasses.replace(m1, **{k: v - h}), target, want_grad=False)[0]
        assert abs(g32[i] / ((Lp - Lm) / (2 * h)) - 1) < 3e-5, k
        h = 1e-2 * v
        Lp = gpu_loss_grad(ev, dataclasses.replace(m1, **{k: v + h}), target, precision="mixed", tol=1e-6,
                           want_grad=False)[0]
        Lm = gpu_loss_grad(ev, dataclasses.replace(m1, **{k: v - h}), target, precision="mixed", tol=1e-6,
                           want_grad=False)[0]
        assert abs(g32[i] / ((Lp - Lm) / (2 * h)) - 1) < 1e-3, k


def test_torch_autograd_function(ev, mat, target):
    import torch
    from paper_1509_04953_gb300.autograd import CurveSetup, stress_strain_curve
    m1 = perturbed(mat)
    g0, q = setup_inputs()
    setup = CurveSetup(N, G, g0, q, mat, SEED, T, -1e-3, 1.0, checkpoint_every=2, adjoint_tol=1e-11)
    theta = torch.tensor([m1.k1, m1.k2, m1.tau0, m1.n], dtype=torch.float64, requires_grad=True)
    curve = stress_strain_curve(theta, setup)
    loss = ((curve - torch.tensor(target)) ** 2).sum()
    loss.backward()
    _, g, _, _ = gpu_loss_grad(ev, m1, target)
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-9, atol=0)


def test_adjoint_on_the_differentiation_workload(ev, mat):
    """32^3, 27 grains, 50 increments (about sqrt(50) = 7 increments per checkpoint): the checkpointed
    FP64 adjoint gradient against central differences of the GPU forward (h = 1e-6 relative)."""
    wl = synth.WORKLOADS["cu32adj"]
    g0 = O.voronoi(wl.n, synth.voronoi_seeds(wl.n, wl.grains, wl.seed))
    q = synth.orientations(wl.grains, wl.seed)
    T = wl.increments

    def run(m, want_grad, target):
        s = ev.Solver(wl.n, wl.grains, g0, q, m, wl.seed, precision="fp64", tol=1e-12, max_iter=40000)
        s.adjoint_begin(T, 7)
        curve = np.array([s.adjoint_step(wl.dE33, wl.dt).sig_mean[2] for _ in range(T)])
        L = float(((curve - target) ** 2).sum()) if target is not None else 0.0
        g = None
        if want_grad:
            gb = np.zeros((T, 6))
            gb[:, 2] = 2 * (curve - target)
            g = s.adjoint_end(gb, tol=1e-11)
        s.close()
        return L, g, curve

    _, _, target = run(mat, False, None)
    m1 = perturbed(mat)
    L, g, _ = run(m1, True, target)
    assert L > 0
    for i, k in enumerate(("k1", "k2", "tau0", "n")):
        v = getattr(m1, k)
        h = 1e-6 * v
        Lp = run(dataclasses.replace(m1, **{k: v + h}), False, target)[0]
        Lm = run(dataclasses.replace(m1, **{k: v - h}), False, target)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(g[i] / fd - 1) < 1e-5, (k, g[i], fd)
