"""Adjoint of the SAIT-preconditioned solve (torch.autograd.Function).

Loss l = 1/2 ||x - x_target||^2 with x = A(kappa)^{-1} b on 3D diffusion with
log-normal kappa (harmonic-mean faces).  Checked against
  * the dense gradient at 8^3: lambda = A^{-T}(x - x_target) from LAPACK,
    dl/db = lambda, dl/dA_ij = -lambda_i x_j;
  * central finite differences (h = 1e-6) on 32 kappa cells and 32 entries of b,
    evaluated with dense solves at 8^3 and with tight GPU solves at 64^3;
  * the transposed SAIT apply against M_L^T (M_U^T g) from the oracle.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

ORDER = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def stencil_masks(N, device):
    idx = torch.arange(N ** 3, device=device)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    valid, nbr = [], []
    for dx, dy, dz in ORDER:
        ok = (x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N) & (z + dz >= 0) & (z + dz < N)
        valid.append(ok)
        nbr.append(torch.where(ok, idx + dx + N * dy + N * N * dz, idx))
    return torch.stack(valid, 1), torch.stack(nbr, 1)


def assemble_values(kappa, valid, nbr):
    """CSR values (synth.varcoef3d's pattern and order) as a differentiable function of kappa."""
    ka = kappa[:, None]
    kb = kappa[nbr]
    face = torch.where(valid, 2 * ka * kb / (ka + kb), ka)     # boundary face: the cell's own kappa
    off = [c for c in range(7) if c != 3]
    diag = face[:, off].sum(1)
    vals = torch.cat([-face[:, :3], diag[:, None], -face[:, 4:]], 1)
    return vals[valid]


@pytest.fixture(scope="module")
def sg():
    from paper_2106_12836_gb300 import build
    build.build()
    import paper_2106_12836_gb300 as m
    return m


def problem(N, seed):
    A = synth.varcoef3d(N, 1.0, seed)
    kappa = np.exp(1.0 * np.random.default_rng(seed).standard_normal(N ** 3))
    b = synth.uniform(seed + 1, A.n)
    xt = synth.uniform(seed + 2, A.n)
    return A, kappa, b, xt


def test_assembly_matches_generator():
    N = 6
    A, kappa, _, _ = problem(N, 3)
    valid, nbr = stencil_masks(N, "cpu")
    vals = assemble_values(torch.from_numpy(kappa), valid, nbr).numpy()
    assert np.allclose(vals, A.va, rtol=1e-14, atol=0)


def loss_grad(sg, ctx, N, kappa_np, b_np, xt_np, opts):
    from paper_2106_12836_gb300.autograd import sait_solve
    A = synth.varcoef3d(N, 1.0, 0)    # pattern only
    valid, nbr = stencil_masks(N, "cuda")
    kappa = torch.tensor(kappa_np, device="cuda", requires_grad=True)
    b = torch.tensor(b_np, device="cuda", requires_grad=True)
    rp = torch.from_numpy(A.rp).cuda()
    ci = torch.from_numpy(A.ci).cuda()
    vals = assemble_values(kappa, valid, nbr)
    vals.retain_grad()
    x = sait_solve(vals, b, rp, ci, ctx, opts)
    loss = 0.5 * ((x - torch.tensor(xt_np, device="cuda")) ** 2).sum()
    loss.backward()
    return (float(loss.detach()), kappa.grad.cpu().numpy(), b.grad.cpu().numpy(), vals.grad.cpu().numpy(),
            x.detach().cpu().numpy())


def dense_loss(N, kappa_np, b_np, xt_np):
    valid, nbr = stencil_masks(N, "cpu")
    A = synth.varcoef3d(N, 1.0, 0)
    vals = assemble_values(torch.from_numpy(kappa_np), valid, nbr).numpy()
    Ad = synth.CSR(A.n, A.rp, A.ci, vals).to_dense()
    x = np.linalg.solve(Ad, b_np)
    return 0.5 * np.sum((x - xt_np) ** 2), Ad, x


def test_dense_gradient_8cubed(sg):
    from paper_2106_12836_gb300.autograd import SolveOptions
    N = 8
    A, kappa, b, xt = problem(N, 11)
    with sg.Context() as ctx:
        opts = SolveOptions(tol=1e-13, restart=60)
        loss, gk, gb, gvals, x = loss_grad(sg, ctx, N, kappa, b, xt, opts)
        torch.cuda.synchronize()
    loss_d, Ad, xd = dense_loss(N, kappa, b, xt)
    lam = np.linalg.solve(Ad.T, xd - xt)
    assert abs(loss - loss_d) <= 1e-10 * abs(loss_d)
    assert np.abs(gb - lam).max() <= 1e-9 * np.abs(lam).max()
    rows = np.repeat(np.arange(A.n), np.diff(A.rp))
    gref = -lam[rows] * xd[A.ci]
    assert np.abs(gvals - gref).max() <= 1e-9 * np.abs(gref).max()
    # central differences on kappa and b with dense solves
    rng = np.random.default_rng(5)
    h = 1e-6
    for c in rng.choice(A.n, 32, replace=False):
        kp, km = kappa.copy(), kappa.copy()
        kp[c] += h
        km[c] -= h
        fd = (dense_loss(N, kp, b, xt)[0] - dense_loss(N, km, b, xt)[0]) / (2 * h)
        assert abs(gk[c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gk).max()), (c, gk[c], fd)
    for c in rng.choice(A.n, 32, replace=False):
        bp, bm = b.copy(), b.copy()
        bp[c] += h
        bm[c] -= h
        fd = (dense_loss(N, kappa, bp, xt)[0] - dense_loss(N, kappa, bm, xt)[0]) / (2 * h)
        assert abs(gb[c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gb).max()), (c, gb[c], fd)


def test_finite_differences_64cubed(sg):
    """Full size (64^3): GPU forward solves to 1e-13 for the differences.

    With iterative solves the loss carries ~cond(A) * tol of noise, so the
    central step is 1e-3 relative to kappa_c here (truncation ~1e-6); the
    h = 1e-6 check runs with dense solves at 8^3 above.
    """
    from paper_2106_12836_gb300.autograd import SolveOptions
    N = 64
    A, kappa, b, xt = problem(N, 21)
    with sg.Context() as ctx:
        opts = SolveOptions(tol=1e-13, restart=50, store="f32")
        loss, gk, gb, _, _ = loss_grad(sg, ctx, N, kappa, b, xt, opts)
        rng = np.random.default_rng(6)
        worst = 0.0
        for c in rng.choice(A.n, 8, replace=False):
            h = 1e-3 * kappa[c]
            kp, km = kappa.copy(), kappa.copy()
            kp[c] += h
            km[c] -= h
            lp = loss_grad(sg, ctx, N, kp, b, xt, opts)[0]
            lm = loss_grad(sg, ctx, N, km, b, xt, opts)[0]
            fd = (lp - lm) / (2 * h)
            worst = max(worst, abs(gk[c] - fd) / max(abs(fd), 1e-3 * np.abs(gk).max()))
        torch.cuda.synchronize()
    assert worst <= 1e-4, worst


def test_transposed_apply(sg, oracle_lib):
    A = synth.convdiff3d(15)
    Lo, Uo = oracle_lib.ilu0(A)
    MLo, MUo = oracle_lib.sait(Lo, 3, "rowrel", 1e-3), oracle_lib.sait(Uo, 3, "rowrel", 1e-3)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with sg.Context() as ctx:
        ML = sg.sait_mat_create_csr(ctx, MLo.n, dev(MLo.rp), dev(MLo.ci), dev(MLo.va))
        MU = sg.sait_mat_create_csr(ctx, MUo.n, dev(MUo.rp), dev(MUo.ci), dev(MUo.va))
        MLT, MUT = sg.sait_mat_transpose(ctx, ML), sg.sait_mat_transpose(ctx, MU)
        T = synth.CSR(MLo.n, *(t.cpu().numpy() for t in MLT.export()))
        assert np.array_equal(T.to_dense(), MLo.to_dense().T)
        P = sg.sait_prec_create_sait(ctx, MUT, MLT)
        g = synth.uniform(3, A.n)
        z = sg.sait_prec_apply(ctx, P, dev(g)).cpu().numpy()
        torch.cuda.synchronize()
    zo = MLo.to_scipy().T @ (MUo.to_scipy().T @ g)
    bound = abs(MLo.to_scipy()).T @ (abs(MUo.to_scipy()).T @ np.abs(g))
    assert np.all(np.abs(z - zo) <= 1e-12 * bound)
