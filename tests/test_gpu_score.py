"""Score-function gradients on the GPU.

Parity: the path statistics (events by class C_k, bit-exact; integrals of N_k,
to 1e-12 relative) and the score against the oracle's run of the same
lattice.  Gradients: the autograd backward (score estimate) against common-
random-number central differences (Delta = 1e-3) within 3 standard errors."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

sr = pytest.importorskip("paper_cs_0405053_gb300")
torch = pytest.importorskip("torch")
from paper_cs_0405053_gb300 import grad  # noqa: E402


def _ends(Tw, n):
    out, t = [], 0.0
    for _ in range(n):
        t = t + Tw
        out.append(t)
    return out


def _check_stats(c, occ, S, ref, J, h, T, glauber):
    assert np.array_equal(c, ref.ev_class.sum(axis=0))
    want = ref.occupancy.sum(axis=0)
    assert np.all(np.abs(occ - want) <= 1e-12 * want.sum()), (occ, want)
    s_ref = oracle.score(ref, J, h, T, glauber)
    scale = np.abs(oracle.score_tables(J, h, T, glauber)[0]).max() * max(1.0, float(c.sum()))
    assert np.all(np.abs(S - s_ref) <= 1e-11 * scale), (S, s_ref)


@pytest.mark.parametrize("L,W,H,T,h,rates,fresh", [
    (32, 8, 8, 1.8, 0.05, "metropolis", False),
    (24, 8, 6, 2.6, -0.1, "glauber", False),
    (16, 4, 4, 3.5, 0.2, "metropolis", True),
    (64, 16, 16, 2.2, 0.0, "metropolis", False)])
def test_score_statistics_match_the_oracle(L, W, H, T, h, rates, fresh):
    lat = sr.Lattice(L, 1.0, h, T, (W, H), seed=L + 3, rates=rates, fresh_steps=fresh, score=True)
    lat.run_windows(0.5, 6)
    c, occ = lat.score_stats()
    S = lat.score()
    ref = oracle.run(L, 1.0, h, T, W, H, L + 3, _ends(0.5, 6), glauber=(rates == "glauber"),
                     fresh_steps=fresh)
    _check_stats(c, occ, S, ref, 1.0, h, T, rates == "glauber")
    # the statistics do not change the trajectory
    assert np.array_equal(lat.spins(), ref.spins[-1])


def test_score_statistics_in_a_batch():
    reps = [dict(L=32, T=2.0, h=0.1, seed=1), dict(L=16, T=3.0, h=-0.2, seed=2, rates="glauber"),
            dict(L=48, T=1.5, h=0.0, seed=3)]
    with sr.Batch(reps, region=(16, 16), score=True) as bt:
        bt.run_adaptive([2.0, 3.0, 1.5], kappa=8.0)
        S = bt.score()
        for b, r in enumerate(reps):
            c, occ = bt.score_stats(b)
            g = r.get("rates") == "glauber"
            ref = oracle.run(r["L"], 1.0, r["h"], r["T"], 16, 16, r["seed"], [bt.t_c[b]], glauber=g)
            _check_stats(c, occ, S[b], ref, 1.0, r["h"], r["T"], g)


def test_gradients_match_common_random_number_differences():
    R, L = 256, 32
    beta, h, J = 0.4, 0.1, 1.0
    spec = grad.AverageSpec(L=[L] * R, seeds=list(range(5000, 5000 + R)), t1=2.0, t2=6.0)
    theta = torch.tensor([[beta, h, J]] * R, dtype=torch.float64, device="cuda",
                         requires_grad=True)
    A = grad.time_averages(theta, spec)
    for j in range(2):                               # m and energy per site
        theta.grad = None
        A[:, j].sum().backward(retain_graph=True)
        g = theta.grad.detach().cpu().numpy()        # per-replica estimates
        est, se = g.mean(axis=0), g.std(axis=0, ddof=1) / math.sqrt(R)
        d = 1e-3
        for q in range(3):
            tp = theta.detach().clone()
            tm = theta.detach().clone()
            tp[:, q] += d
            tm[:, q] -= d
            Ap = grad._simulate(tp.cpu().numpy(), spec)[0][:, j]
            Am = grad._simulate(tm.cpu().numpy(), spec)[0][:, j]
            fd = (Ap - Am) / (2 * d)
            fd_mean, fd_se = fd.mean(), fd.std(ddof=1) / math.sqrt(R)
            tol = 3.0 * math.hypot(se[q], fd_se)
            assert abs(est[q] - fd_mean) <= tol, (j, q, est[q], se[q], fd_mean, fd_se)


def test_grad_kernel_matches_its_definition():
    """sr_score_grad against the formula evaluated on the host."""
    rng = np.random.default_rng(1)
    n, m, nq = 37, 2, 3
    A, gA, S = rng.normal(size=(n, m)), rng.normal(size=(n, m)), rng.normal(size=(n, nq))
    E = rng.normal(size=(n, m, nq))
    dev = [torch.from_numpy(x).cuda() for x in (A, gA, S, E)]
    G = torch.empty((n, nq), dtype=torch.float64, device="cuda")
    lib = sr.library()
    rc = lib.sr_score_grad(n, m, nq, *[x.data_ptr() for x in dev], G.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    base = (A.sum(axis=0)[None, :] - A) / (n - 1)
    want = np.einsum("ij,ijq->iq", gA, (A - base)[:, :, None] * S[:, None, :] + E)
    assert np.allclose(G.cpu().numpy(), want, rtol=1e-12, atol=1e-12)


def _fd(theta, spec, q, j, d=1e-3):
    tp, tm = theta.detach().clone(), theta.detach().clone()
    tp[:, q] += d
    tm[:, q] -= d
    ap = grad._simulate(tp.cpu().numpy(), spec)[0][:, j]
    am = grad._simulate(tm.cpu().numpy(), spec)[0][:, j]
    return (ap - am) / (2 * d)


@pytest.mark.parametrize("h", [0.0, 0.05])
def test_c5_shaped_gradients_at_and_off_the_kink(h):
    """The differentiation workload's shape at a smaller size: 128 replicas
    of L = 256 at T = 2.8 from fair-coin spins, time averages of m and the
    energy per site over t in [40, 100].  All six score-function derivatives
    (d/d(beta, h, J) of both averages) against common-random-number central
    differences (Delta = 1e-3) within 3.5 combined standard errors.  At h = 0
    the n_up = 2 classes sit on the kink of the Metropolis rate (the score
    takes the mean of the one-sided derivatives there).  At h = 0 also the
    fluctuation relation d<m>/dh = beta N Var(m) (N = L^2, the variance of the
    instantaneous m over the independent replicas): the chain is in
    equilibrium over the averaging interval, so the central difference of the
    time average must agree with it within 4 standard errors (jackknife over
    replicas for the variance)."""
    R, L, T = 128, 256, 2.8
    beta = 1.0 / T
    spec = grad.AverageSpec(L=[L] * R, seeds=list(range(9000, 9000 + R)), t1=40.0, t2=100.0)
    theta = torch.tensor([[beta, h, 1.0]] * R, dtype=torch.float64, device="cuda",
                         requires_grad=True)
    A = grad.time_averages(theta, spec)
    zs = []
    fd_dmdh = None
    for j in range(2):
        theta.grad = None
        A[:, j].sum().backward(retain_graph=True)
        g = theta.grad.detach().cpu().numpy()
        est, se = g.mean(axis=0), g.std(axis=0, ddof=1) / math.sqrt(R)
        for q in range(3):
            fd = _fd(theta, spec, q, j)
            z = (est[q] - fd.mean()) / math.hypot(se[q], fd.std(ddof=1) / math.sqrt(R))
            zs.append(z)
            if (j, q) == (0, 1):
                fd_dmdh = fd
    assert max(abs(z) for z in zs) <= 3.5, zs
    if h == 0.0:
        _, _, _, ms = grad._simulate(theta.detach().cpu().numpy(), spec, samples=30)
        var = ms.var(axis=0, ddof=1).mean()
        jack = np.array([np.delete(ms, i, axis=0).var(axis=0, ddof=1).mean() for i in range(R)])
        se_var = math.sqrt((R - 1) / R * ((jack - jack.mean()) ** 2).sum())
        rel = beta * L * L * var
        se_rel = beta * L * L * se_var
        z = (fd_dmdh.mean() - rel) / math.hypot(fd_dmdh.std(ddof=1) / math.sqrt(R), se_rel)
        assert abs(z) <= 4.0, (fd_dmdh.mean(), rel, z)
