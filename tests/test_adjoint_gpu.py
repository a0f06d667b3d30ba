"""The adjoint of the time step on the GPU (rlb_record / rlb_backward / rlb_moments_vjp / rlb_fields_vjp /
rlb_init_vjp and the torch.autograd wrapper) against central differences of the GPU forward, against the
oracle's central-difference gradient, against closed forms, and for checkpoint independence.

Loss used throughout: L(M) = sum_a,x R_a(x) M_a(x) + 1/2 sum_x T^xx(x)^2 of the five conserved moments M after
the run, R seeded. Differences: along a rough (per-cell random) direction the WENO5 limiter makes the loss
strongly curved on the scale of a 1e-5 perturbation (measured with the oracle on the ballistic case below:
fourth-order differences give 6.4682 at h = 1e-5, 6.46805612 at 1e-6 and 6.46805610 at 1e-7, while along a
smooth direction they agree to 1e-10 from h = 1e-5 down). Along rough directions the tests therefore use the
fourth-order difference (8 (f(h) - f(-h)) - (f(2h) - f(-2h))) / 12h at h = 1e-7 (rounding ~1e-9 |L|); the
single-parameter differences (log tau, one cell) use the second-order one at h = 1e-6. Adjoint and difference
must agree to 1e-6 relative or 1e-8 |L|, whichever is larger.
"""
import math

import numpy as np
import pytest
import torch

import harness as H
import oracle
from oracle import gradient as og
from paper_1608_03004_gb300 import adjoint
from paper_1608_03004_gb300 import binding as rb
from paper_1608_03004_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


def smooth_fields(Nx, seed, vmax=0.3):
    rng = np.random.default_rng(seed)
    x = (np.arange(Nx) + 0.5) / Nx
    P = 1.0 + 0.25 * np.sin(2 * np.pi * x + rng.uniform(0, 6)) + 0.1 * np.cos(6 * np.pi * x + rng.uniform(0, 6))
    n = 1.0 + 0.2 * np.cos(2 * np.pi * x + rng.uniform(0, 6))
    v = vmax * np.sin(4 * np.pi * x + rng.uniform(0, 6))
    return P, n, v


def make_tube(Nx, Qxi, tau, bc, dt=None):
    return rb.Tube.make(Nx, Qxi, tau, dt=0.5 / Nx if dt is None else dt, bc=bc)


def with_tau(t, tau):
    return rb.Tube(t.Qp, t.Qxi, t.Np, t.Nv, t.Nx, t.dx, t.dt, tau, t.bc, t.storage)


def loss_np(M, R):
    return float(np.sum(R * M) + 0.5 * np.sum(M[4] ** 2))


def forward(tubes, P, n, v, nsteps):
    with rb.rlb_init(tubes, P, n, v) as h:
        rb.rlb_step(h, nsteps)
        return rb.rlb_moments(h)[:5].copy()


def forward_fields(tubes, P, n, v, nsteps):
    with rb.rlb_init(tubes, P, n, v) as h:
        rb.rlb_step(h, nsteps)
        return rb.rlb_moments(h).copy()


def adjoint_grads(tubes, P, n, v, nsteps, every, R):
    lt = torch.tensor([math.log(t.tau) if math.isfinite(t.tau) else math.inf for t in tubes], dtype=torch.float64,
                      requires_grad=True)
    Pt, nt, vt = (torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=True) for a in (P, n, v))
    M = adjoint.run_moments(lt, Pt, nt, vt, tubes, nsteps, every)
    Rt = torch.tensor(R, device=DEV)
    L = (Rt * M).sum() + 0.5 * (M[4] ** 2).sum()
    L.backward()
    return (float(L.detach()), lt.grad.numpy().copy(), Pt.grad.cpu().numpy(), nt.grad.cpu().numpy(),
            vt.grad.cpu().numpy())


def fd4(f, h=1e-7):
    """Fourth-order central difference of f(s) at s = 0."""
    return (8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)


def close(adj, fd, L, rel=1e-6, absL=1e-8):
    return abs(adj - fd) <= rel * abs(fd) + absL * abs(L)


@pytest.fixture(scope="module")
def batch():
    t0 = make_tube(150, 8, 0.02, W.BC_PERIODIC)
    t1 = make_tube(200, 16, 0.05, W.BC_OPEN)
    P0, n0, v0 = smooth_fields(150, 1)
    b = W.gaussian_bumps(Nx=200, Qxi=16, tau=0.05, seed=7)
    P = np.concatenate([P0, b.P])
    n = np.concatenate([n0, b.n])
    v = np.concatenate([v0, 0.1 * np.sin(np.linspace(0, 3, 200))])
    R = np.random.default_rng(3).normal(size=(5, 350))
    return [t0, t1], P, n, v, R


def test_log_tau_gradients_match_central_differences(batch):
    tubes, P, n, v, R = batch
    nsteps, h = 60, 1e-6
    L, glt, *_ = adjoint_grads(tubes, P, n, v, nsteps, 16, R)
    assert L == pytest.approx(loss_np(forward(tubes, P, n, v, nsteps), R), rel=1e-14)
    for b in range(2):
        lp = [with_tau(t, t.tau * math.exp(h)) if k == b else t for k, t in enumerate(tubes)]
        lm = [with_tau(t, t.tau * math.exp(-h)) if k == b else t for k, t in enumerate(tubes)]
        fd = (loss_np(forward(lp, P, n, v, nsteps), R) - loss_np(forward(lm, P, n, v, nsteps), R)) / (2 * h)
        print(f"tube {b}: dL/dlog tau adjoint {glt[b]:.12e} central difference {fd:.12e}")
        assert close(glt[b], fd, L), (b, glt[b], fd)


def test_field_gradients_match_directional_differences(batch):
    tubes, P, n, v, R = batch
    nsteps = 60
    L, _, gP, gn, gv = adjoint_grads(tubes, P, n, v, nsteps, 16, R)
    rng = np.random.default_rng(11)
    for _ in range(3):
        dP, dn, dv = (rng.normal(size=P.size) for _ in range(3))
        dv *= 0.5
        fd = fd4(lambda s: loss_np(forward(tubes, P + s * dP, n + s * dn, v + s * dv, nsteps), R))
        adj = float(np.dot(gP, dP) + np.dot(gn, dn) + np.dot(gv, dv))
        print(f"directional derivative: adjoint {adj:.12e} central difference {fd:.12e}")
        assert close(adj, fd, L), (adj, fd)


def test_gradients_match_the_oracle():
    """Open tube of 40 cells (the boundary cells included) against the oracle's central differences."""
    Nx, Qxi, tau, nsteps = 40, 8, 0.04, 24
    t = make_tube(Nx, Qxi, tau, W.BC_OPEN)
    P, n, v = smooth_fields(Nx, 5, vmax=0.2)
    R = np.random.default_rng(8).normal(size=(5, Nx))
    L, glt, gP, gn, gv = adjoint_grads([t], P, n, v, nsteps, 7, R)
    p = oracle.params(Qxi=Qxi, Nx=Nx, tau=tau, dt=t.dt, bc=oracle.BC_OPEN)
    loss = lambda m: loss_np(m, R)  # noqa: E731
    g_or = og.grad_log_tau(p, P, n, v, nsteps, loss)
    print(f"dL/dlog tau: adjoint {glt[0]:.12e} oracle {g_or:.12e}")
    assert close(glt[0], g_or, L)
    cells = [0, 1, 13, 38, 39]
    for which, g in (("P", gP), ("n", gn), ("v", gv)):
        ref = og.grad_field(p, P, n, v, nsteps, loss, which, cells)
        for k, x in enumerate(cells):
            assert close(g[x], ref[k], L), (which, x, g[x], ref[k])


def test_conserved_sums(batch):
    """Periodic tube, loss sum_x T^00: dL/dP = 4 gamma^2 - 1, dL/dn = 0, dL/dv = 8 P gamma^4 v, dL/dlog tau = 0
    (T^00 = (4 gamma^2 - 1) P initially, and conserved)."""
    tubes, P, n, v, _ = batch
    t = tubes[0]
    Pp, n_, vp = P[:150], n[:150], v[:150]
    lt = torch.tensor([math.log(t.tau)], dtype=torch.float64, requires_grad=True)
    Pt, nt, vt = (torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=True) for a in (Pp, n_, vp))
    M = adjoint.run_moments(lt, Pt, nt, vt, [t], 40, 9)
    M[2].sum().backward()
    g2 = 1.0 / (1.0 - vp**2)
    np.testing.assert_allclose(Pt.grad.cpu().numpy(), 4 * g2 - 1, rtol=1e-10)
    np.testing.assert_allclose(nt.grad.cpu().numpy(), 0.0, atol=1e-10)
    np.testing.assert_allclose(vt.grad.cpu().numpy(), 8 * Pp * g2 * g2 * vp, rtol=1e-9, atol=1e-10)
    assert abs(float(lt.grad[0])) < 1e-9 * float(M[2].sum().detach())


def test_uniform_relaxation_closed_form():
    """Uniform state at rest, anisotropic but even in xi: F - F^eq shrinks by R(-dt/tau) per step, so
    dT^xx_N/dlog tau = (T^xx_0 - T^00/3) N R^(N-1) R'(z) dt/tau per cell."""
    Nx, Qxi, tau, N = 10, 8, 0.03, 8
    t = make_tube(Nx, Qxi, tau, W.BC_PERIODIC, dt=0.01)
    _, _, xi, _ = rb.rlb_quadrature(3, Qxi)
    with rb.rlb_init([t], np.full(Nx, 1.04), np.full(Nx, 0.8), np.zeros(Nx)) as h:
        F = rb.rlb_get_state(h).reshape(3 * Qxi, Nx)
        F = F * (1.0 + 0.08 * np.tile(0.5 * (3 * xi**2 - 1), 3))[:, None]
        rb.rlb_set_state(h, F)
        m0 = rb.rlb_moments(h)
        rb.rlb_record(h, N, 3)
        gm = torch.zeros((5, Nx), dtype=torch.float64, device=DEV)
        gm[4] = 1.0
        seed = torch.empty(3 * Qxi * Nx, dtype=torch.float64, device=DEV)
        rb.rlb_moments_vjp(h, gm, seed)
        _, glt = rb.rlb_backward(h, seed)
    z = -t.dt / tau
    R, dR = 1 + z + z * z / 2 + z**3 / 6, 1 + z + z * z / 2
    exact = float(np.sum(m0[4] - m0[2] / 3.0)) * N * R ** (N - 1) * dR * (t.dt / tau)
    assert glt[0] == pytest.approx(exact, rel=1e-10)


def test_checkpoint_interval_does_not_change_the_gradient(batch):
    tubes, P, n, v, R = batch
    ref = None
    for every in (1, 5, 23, 40):
        _, glt, gP, gn, gv = adjoint_grads(tubes, P, n, v, 23, every, R)
        cur = np.concatenate([glt, gP, gn, gv])
        if ref is None:
            ref = cur
        else:
            np.testing.assert_array_equal(cur, ref, err_msg=f"every={every}")


def test_ballistic_tube():
    """tau = infinity: no relaxation-time gradient; the field gradients still match differences."""
    Nx, nsteps = 120, 50
    t = make_tube(Nx, 16, math.inf, W.BC_PERIODIC)
    P, n, v = smooth_fields(Nx, 9)
    R = np.random.default_rng(4).normal(size=(5, Nx))
    L, glt, gP, gn, gv = adjoint_grads([t], P, n, v, nsteps, 10, R)
    assert glt[0] == 0.0
    dP = np.random.default_rng(2).normal(size=Nx)
    fd = fd4(lambda s: loss_np(forward([t], P + s * dP, n, v, nsteps), R))
    print(f"ballistic directional derivative: adjoint {float(np.dot(gP, dP)):.12e} difference {fd:.12e}")
    assert close(float(np.dot(gP, dP)), fd, L)


def test_reduced_storage_and_missing_record_rejected():
    t = rb.Tube.make(64, 8, 1e-2, storage=rb.STORAGE_F32)
    with rb.rlb_init([t], np.ones(64), np.ones(64), np.zeros(64)) as h:
        with pytest.raises(rb.RlbError) as ei:
            rb.rlb_record(h, 3, 1)
        assert ei.value.status == rb.EINVAL
    t = make_tube(64, 8, 1e-2, W.BC_OPEN)
    with rb.rlb_init([t], np.ones(64), np.ones(64), np.zeros(64)) as h:
        seed = torch.zeros(h.state_size, dtype=torch.float64, device=DEV)
        with pytest.raises(rb.RlbError) as ei:
            rb.rlb_backward(h, seed)
        assert ei.value.status == rb.EINVAL
        with pytest.raises(rb.RlbError):
            rb.rlb_record(h, 0, 1)


def test_fields_vjp_matches_differences_of_the_oracle_fields():
    """rlb_fields_vjp at a state off equilibrium (a smooth flow at |v| up to 0.6 stepped 5 times): for
    L = sum_{f,x} g_f(x) field_f(x) over all eight fields, its seed dotted with a direction dF equals the
    central difference of the oracle's fields along dF (the fields are smooth functions of F: the moment sums,
    then the Landau-frame closed form), to 1e-8."""
    s = W.random_smooth(96, 8, 2e-2, seed=21, vmax=0.6)
    p = H.to_params(s)
    F = oracle.step(p, H.oracle_init(s), 5)
    rng = np.random.default_rng(22)
    g = rng.normal(size=(rb.NFIELDS, s.Nx))
    with H.gpu_init([s]) as h:
        rb.rlb_set_state(h, F.ravel())
        seed = torch.empty(h.state_size, dtype=torch.float64, device=DEV)
        rb.rlb_fields_vjp(h, torch.tensor(g, device=DEV), seed)
        seed = seed.cpu().numpy().reshape(s.Q, s.Nx)
    scale = np.max(np.abs(F), axis=1, keepdims=True)
    for _ in range(3):
        dF = rng.normal(size=F.shape) * scale
        hstep = 1e-6
        fd = (np.sum(g * oracle.fields(p, F + hstep * dF)) - np.sum(g * oracle.fields(p, F - hstep * dF))) / (2 * hstep)
        adj = float(np.sum(seed * dF))
        print(f"fields vjp: adjoint {adj:.12e} oracle difference {fd:.12e}")
        assert abs(adj - fd) <= 1e-8 * abs(fd), (adj, fd)


def energy_loss(f, R):
    """Loss of all the fields: sum_x R_e e + R_v v + R_n n + 1/2 sum_x e^2."""
    return float(np.sum(R[0] * f[5] + R[1] * f[6] + R[2] * f[7]) + 0.5 * np.sum(f[5] ** 2))


def test_energy_loss_gradients_match_the_oracle():
    """A loss of the Landau-frame e, v, n through rlb_fields_vjp and the torch wrapper: open tube of 40 cells
    against the oracle's central differences in log tau and at cells (the boundary cells included)."""
    Nx, Qxi, tau, nsteps = 40, 8, 0.04, 24
    t = make_tube(Nx, Qxi, tau, W.BC_OPEN)
    P, n, v = smooth_fields(Nx, 6, vmax=0.3)
    R = np.random.default_rng(9).normal(size=(3, Nx))
    lt = torch.tensor([math.log(tau)], dtype=torch.float64, requires_grad=True)
    Pt, nt, vt = (torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=True) for a in (P, n, v))
    f = adjoint.run_fields(lt, Pt, nt, vt, [t], nsteps, 7)
    Rt = torch.tensor(R, device=DEV)
    L = (Rt[0] * f[5] + Rt[1] * f[6] + Rt[2] * f[7]).sum() + 0.5 * (f[5] ** 2).sum()
    L.backward()
    L = float(L.detach())
    p = oracle.params(Qxi=Qxi, Nx=Nx, tau=tau, dt=t.dt, bc=oracle.BC_OPEN)
    loss = lambda m: energy_loss(m, R)  # noqa: E731
    assert L == pytest.approx(loss(og.run_moments(p, P, n, v, nsteps, rows=8)), rel=1e-13)
    g_or = og.grad_log_tau(p, P, n, v, nsteps, loss, rows=8)
    print(f"e, v, n loss: dL/dlog tau adjoint {float(lt.grad[0]):.12e} oracle {g_or:.12e}")
    assert close(float(lt.grad[0]), g_or, L, absL=1e-9)
    cells = [0, 1, 17, 38, 39]
    for which, g in (("P", Pt.grad), ("n", nt.grad), ("v", vt.grad)):
        g = g.cpu().numpy()
        ref = og.grad_field(p, P, n, v, nsteps, loss, which, cells, rows=8)
        for k, x in enumerate(cells):
            assert close(g[x], ref[k], L, absL=1e-9), (which, x, g[x], ref[k])


def test_gradient_workload_full_size():
    """The inverse problem on Gaussian bumps at full size (Nx = 2048, Q = 3 x 32, 1000 steps, checkpoints every
    50): the loss is the squared L2 distance of the final energy density e(x) to a target produced by a run with
    tau* = 0.05 from the initial pressure perturbed by a second seed-fixed set of Gaussian bumps (amplitude
    0.05); its gradient in log tau and in the initial P(x), at tau = 0.08 and the unperturbed P, against
    central differences (h = 1e-6) of the GPU forward."""
    spec = W.gaussian_bumps()
    tgt = W.perturbed(spec, seed=5)
    nsteps, every, h = 1000, 50, 1e-6
    t_star = rb.Tube.make(spec.Nx, spec.Qxi, 0.05, dt=spec.dt, dx=spec.dx)
    target = forward_fields([t_star], tgt.P, tgt.n, tgt.v, nsteps)[5]
    t = with_tau(t_star, 0.08)

    def loss_t(f):
        return 0.5 * float(np.sum((f[5] - target) ** 2))

    lt = torch.tensor([math.log(0.08)], dtype=torch.float64, requires_grad=True)
    Pt, nt, vt = (torch.tensor(a, dtype=torch.float64, device=DEV, requires_grad=True)
                  for a in (spec.P, spec.n, spec.v))
    f = adjoint.run_fields(lt, Pt, nt, vt, [t], nsteps, every)
    L = 0.5 * ((f[5] - torch.tensor(target, device=DEV)) ** 2).sum()
    L.backward()
    fd = (loss_t(forward_fields([with_tau(t, 0.08 * math.exp(h))], spec.P, spec.n, spec.v, nsteps))
          - loss_t(forward_fields([with_tau(t, 0.08 * math.exp(-h))], spec.P, spec.n, spec.v, nsteps))) / (2 * h)
    g = float(lt.grad[0])
    print(f"full size: L = {float(L):.6e}, dL/dlog tau adjoint {g:.10e} central difference {fd:.10e}")
    assert close(g, fd, float(L), rel=1e-5, absL=1e-9)
    gP = Pt.grad.cpu().numpy()
    for x in (300, 1024, 1700):
        Pp, Pm = spec.P.copy(), spec.P.copy()
        Pp[x] += h
        Pm[x] -= h
        fdx = (loss_t(forward_fields([t], Pp, spec.n, spec.v, nsteps))
               - loss_t(forward_fields([t], Pm, spec.n, spec.v, nsteps))) / (2 * h)
        print(f"  dL/dP({x}): adjoint {gP[x]:.10e} central difference {fdx:.10e}")
        assert close(gP[x], fdx, float(L), rel=1e-5, absL=1e-9), (x, gP[x], fdx)


@pytest.mark.parametrize("Qp,Np,Nv,Qxi,bc", [(4, 3, 8, 6, W.BC_OPEN), (3, 2, 5, 7, W.BC_PERIODIC),
                                             (4, 2, 5, 5, W.BC_OPEN)])
def test_other_orders_match_central_differences(Qp, Np, Nv, Qxi, bc):
    """The adjoint kernel's generic instantiation (Np = 3, Nv = 8), odd Qxi (a xi = 0 node, no advection) and
    four radial nodes: dL/dlog tau by second-order differences, a smooth direction in (P, n, v) by fourth-order
    ones (h = 1e-5: smooth directions converge there)."""
    Nx, nsteps = 90, 30
    t = rb.Tube.make(Nx, Qxi, 0.03, dt=0.5 / Nx, bc=bc, Qp=Qp, Np=Np, Nv=Nv)
    P, n, v = smooth_fields(Nx, Qp * 10 + Qxi, vmax=0.3)
    R = np.random.default_rng(Qxi).normal(size=(5, Nx))
    L, glt, gP, gn, gv = adjoint_grads([t], P, n, v, nsteps, 8, R)
    h = 1e-6
    fd = (loss_np(forward([with_tau(t, t.tau * math.exp(h))], P, n, v, nsteps), R)
          - loss_np(forward([with_tau(t, t.tau * math.exp(-h))], P, n, v, nsteps), R)) / (2 * h)
    print(f"Qp={Qp} Np={Np} Nv={Nv} Qxi={Qxi}: dL/dlog tau adjoint {glt[0]:.12e} difference {fd:.12e}")
    assert close(glt[0], fd, L)
    x = (np.arange(Nx) + 0.5) / Nx
    dP, dn, dv = np.sin(2 * np.pi * x), np.cos(4 * np.pi * x), 0.3 * np.sin(2 * np.pi * x + 1.0)
    fdd = fd4(lambda s: loss_np(forward([t], P + s * dP, n + s * dn, v + s * dv, nsteps), R), h=1e-5)
    adj = float(np.dot(gP, dP) + np.dot(gn, dn) + np.dot(gv, dv))
    print(f"  directional: adjoint {adj:.12e} difference {fdd:.12e}")
    assert close(adj, fdd, L)
