"""The differentiable solve on the GPU: gradient kernels against the oracle,
value updates of a handle, and the autograd chain (coefficients -> stored
values -> solution -> loss L = ||x - x_t||^2) against dense reference
gradients and central finite differences.

Gates:
  - gradient kernels: per entry within a few roundings of the oracle's value
    (each is one or two products, or a short fixed-order sum);
  - 6x6x6 grid: gradients with respect to b, the stored values (full and
    symmetric storage) and the element coefficients within 1e-8 (relative,
    2-norm) of the dense-solve reference;
  - 64x64x64 grid: 32 random directions -- relative white noise
    (r * |theta|, r ~ N(0, I)) in b and the stored values, random smooth
    fields times c_e in the element coefficients -- fourth-order central
    differences with step 1e-6 of a fixed-iteration solve (a smooth map),
    relative error <= 1e-5.
"""
import numpy as np
import pytest

import femgen
import oracle
import paper_1010_4639_gb300 as gb

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def torch():
    import torch
    gb.build()
    assert torch.cuda.is_available()
    return torch


def arrays(s, fmt):
    return {"csr": (s.ptr, s.idx, s.val), "sym": s.upper(), "csc": s.csc()}[fmt]


@pytest.mark.parametrize("fmt", ["csr", "csc", "sym"])
def test_grad_values_kernel_matches_oracle(torch, fmt):
    s = femgen.build_system(femgen.Grid(17, 15, 19, seed_mesh=2, seed_x=3))
    ptr, idx, val = arrays(s, fmt)
    lam = femgen.random_vector(s.n, 5)
    x = femgen.random_vector(s.n, 6)
    g = gb.grad_values(fmt, torch.from_numpy(ptr).cuda(), torch.from_numpy(idx).cuda(),
                       torch.from_numpy(lam).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.grad_values(fmt, ptr, idx, lam, x)
    rows = np.repeat(np.arange(s.n), np.diff(ptr))
    scale = np.abs(lam[rows] * x[idx]) + np.abs(lam[idx] * x[rows])
    assert np.all(np.abs(g - ref) <= 4 * EPS * scale)


def test_element_kernels_match_oracle(torch):
    g = femgen.Grid(12, 13, 11, seed_mesh=4, seed_x=5)
    s = femgen.build_system(g)
    el = femgen.elements(g)
    for storage, (pp, ii, vv) in (("csr", (s.ptr, s.idx, s.val)), ("sym", s.upper())):
        pos, w = femgen.element_map(el, pp, ii, storage=storage)
        tptr, te, tw = femgen.assembly_map(pos, w, len(ii))
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        val = gb.assemble(T(tptr), T(te), T(tw), T(el.coef)).cpu().numpy()
        ref = oracle.assemble(tptr, te, tw, el.coef)
        bound = np.array([np.abs(tw[tptr[p]:tptr[p + 1]] * el.coef[te[tptr[p]:tptr[p + 1]]]).sum()
                          for p in range(len(ii))])
        assert np.all(np.abs(val - ref) <= 16 * EPS * bound)
        gv = femgen.random_vector(len(ii), 9)
        gc = gb.element_grad(T(pos), T(w), T(gv)).cpu().numpy()
        refc = oracle.element_grad(pos, w, gv)
        boundc = np.abs(w * np.where(pos >= 0, gv[np.maximum(pos, 0)], 0.0)).sum(axis=1)
        assert np.all(np.abs(gc - refc) <= 32 * EPS * boundc)


@pytest.mark.parametrize("fmt", ["csr", "csc", "sym"])
def test_update_values_equals_a_fresh_handle(torch, fmt):
    g = femgen.Grid(20, 18, 21, seed_mesh=6, seed_x=7)
    s = femgen.build_system(g)
    ptr, idx, val = arrays(s, fmt)
    rng = np.random.default_rng(3)
    new = val * rng.uniform(0.5, 1.5, val.shape[0])
    if fmt != "sym":  # keep the full matrix symmetric: scale (i, j) and (j, i) alike
        rows = np.repeat(np.arange(s.n), np.diff(ptr))
        f = 1.0 + 0.5 * np.sin(np.minimum(rows, idx) * 7.0 + np.maximum(rows, idx) * 3.0)
        new = val * f
    x = torch.from_numpy(femgen.random_vector(s.n, 8)).cuda()
    with gb.Matrix(fmt, ptr, idx, val) as A, gb.Matrix(fmt, ptr, idx, new) as F:
        A.update_values(torch.from_numpy(new).cuda())
        assert torch.equal(A.spmv(x), F.spmv(x))
        assert torch.equal(A.spmv_f32(x.float()), F.spmv_f32(x.float()))
        A.update_values(val)  # host memory, back to the original
        with gb.Matrix(fmt, ptr, idx, val) as O:
            assert torch.equal(A.spmv(x), O.spmv(x))


def dense_reference(s, el, xt):
    A = np.zeros((s.n, s.n))
    for i in range(s.n):
        A[i, s.idx[s.ptr[i]:s.ptr[i + 1]]] = s.val[s.ptr[i]:s.ptr[i + 1]]
    x = np.linalg.solve(A, s.b)
    lam = np.linalg.solve(A, 2.0 * (x - xt))
    GA = -np.outer(lam, x)
    ok = el.nodes >= 0
    safe = np.where(ok, el.nodes, 0)
    Gsub = GA[safe[:, :, None], safe[:, None, :]] * (ok[:, :, None] & ok[:, None, :])
    return x, lam, GA, np.einsum("eab,eab->e", el.kh, Gsub)


def chain(torch, s, el, fmt, **kw):
    """coef -> values -> x -> L on the GPU; returns (L, x, grad_b, grad_values, grad_coef)."""
    pp, ii, _ = arrays(s, fmt)
    storage = "sym" if fmt == "sym" else "csr"
    pos, w = femgen.element_map(el, pp, ii, storage=storage)
    tptr, te, tw = femgen.assembly_map(pos, w, len(ii))
    asm = gb.Assembly(pos, w, tptr, te, tw)
    coef = torch.from_numpy(el.coef.copy()).cuda().requires_grad_(True)
    vals = asm(coef)
    vals.retain_grad()
    S = gb.SparseSolve(fmt, pp, ii, vals.detach().cpu().numpy(), **kw)
    b = torch.from_numpy(s.b.copy()).cuda().requires_grad_(True)
    return S, asm, coef, vals, b, (pos, w, tptr, te, tw)


def test_autograd_matches_dense_reference(torch):
    g = femgen.Grid(6, 6, 6, contrast=50.0, seed_mesh=7, seed_x=8)
    s = femgen.build_system(g)
    el = femgen.elements(g)
    xt = femgen.random_vector(s.n, 77)
    x_ref, lam_ref, GA, gc_ref = dense_reference(s, el, xt)
    rows = np.repeat(np.arange(s.n), np.diff(s.ptr))
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    for fmt in ("csr", "sym"):
        S, asm, coef, vals, b, _ = chain(torch, s, el, fmt, tol=1e-13)
        x = S(vals, b)
        L = ((x - torch.from_numpy(xt).cuda()) ** 2).sum()
        L.backward()
        assert rel(x.detach().cpu().numpy(), x_ref) <= 1e-10
        assert rel(b.grad.cpu().numpy(), lam_ref) <= 1e-8
        gv = vals.grad.cpu().numpy()
        if fmt == "csr":
            assert rel(gv, GA[rows, s.idx]) <= 1e-8
        else:
            up, ui, _ = s.upper()
            ur = np.repeat(np.arange(s.n), np.diff(up))
            assert rel(gv, np.where(ur == ui, GA[ur, ui], GA[ur, ui] + GA[ui, ur])) <= 1e-8
        assert rel(coef.grad.cpu().numpy(), gc_ref) <= 1e-8
        S.close()


def test_autograd_matches_oracle_gradients(torch):
    g = femgen.Grid(12, 12, 12, contrast=1000.0, seed_mesh=9, seed_x=10)
    s = femgen.build_system(g)
    el = femgen.elements(g)
    xt = femgen.random_vector(s.n, 78)
    S, asm, coef, vals, b, (pos, w, *_rest) = chain(torch, s, el, "sym", tol=1e-13)
    x = S(vals, b)
    L = ((x - torch.from_numpy(xt).cuda()) ** 2).sum()
    L.backward()
    up, ui, _ = s.upper()
    Lo, xo, lamo, gbo, gvo = oracle.loss_gradients("sym", up, ui, vals.detach().cpu().numpy(), s.b, xt, tol=1e-13)
    gco = oracle.element_grad(pos, w, gvo)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)  # noqa: E731
    assert abs(float(L.detach()) - Lo) <= 1e-9 * Lo
    assert rel(b.grad.cpu().numpy(), gbo) <= 1e-8
    assert rel(vals.grad.cpu().numpy(), gvo) <= 1e-8
    assert rel(coef.grad.cpu().numpy(), gco) <= 1e-8
    S.close()


def smooth_field(torch, g, gen):
    """Random low-frequency field on the elements of grid g (one value per tetrahedron)."""
    e = torch.arange(6 * (g.nx - 1) * (g.ny - 1) * (g.nz - 1), device="cuda") // 6
    ci = (e % (g.nx - 1)).double()
    cj = ((e // (g.nx - 1)) % (g.ny - 1)).double()
    ck = (e // ((g.nx - 1) * (g.ny - 1))).double()
    p = torch.stack([(ci + 0.5) / (g.nx - 1), (cj + 0.5) / (g.ny - 1), (ck + 0.5) / (g.nz - 1)], dim=1)
    f = torch.zeros(e.shape[0], dtype=torch.float64, device="cuda")
    for _ in range(3):
        k = torch.randint(0, 3, (3,), generator=gen, device="cuda").double()
        a = torch.randn((), generator=gen, device="cuda", dtype=torch.float64)
        ph = 6.283185307179586 * torch.rand((), generator=gen, device="cuda", dtype=torch.float64)
        f += a * torch.cos(6.283185307179586 * (p @ k) + ph)
    return f


def test_finite_differences_64(torch):
    """The differentiation configuration: 64^3 grid, L = ||x - x_t||^2,
    32 random relative directions (11 in b, 11 in the stored values, 10 in
    the element coefficients), central differences with step 1e-6."""
    g = femgen.DIFF
    s = femgen.build_system(g)
    el = femgen.elements(g)
    xt = torch.from_numpy(femgen.random_vector(s.n, 79)).cuda()
    # iterations for a 1e-13 residual, then every solve runs exactly that many
    up, ui, uv = s.upper()
    with gb.Matrix("sym", up, ui, uv) as A:
        _, info = A.solve(torch.from_numpy(s.b).cuda(), tol=1e-13, maxit=100000)
    assert info.status == "OK"
    K = info.iterations + 50
    S, asm, coef, vals, b, _ = chain(torch, s, el, "sym", fixed_iterations=K)
    x = S(vals, b)
    L = ((x - xt) ** 2).sum()
    L.backward()
    gb_, gv, gc = b.grad.clone(), vals.grad.clone(), coef.grad.clone()

    def solution(v, bb):
        with torch.no_grad():
            return S(v, bb)

    def diff(vp, bp, vm, bm):
        # L(+) - L(-) summed as (x+ - x-) . (x+ + x- - 2 x_t): the same
        # difference without cancelling two losses of size ~n
        xp, xm = solution(vp, bp), solution(vm, bm)
        return float(((xp - xm) * (xp + xm - 2.0 * xt)).sum())

    def derivative(point, step=None):
        # fourth-order central stencil with step h: its truncation error is
        # O(h^4); the second-order stencil's O(h^2) term exceeds 1e-5 on the
        # stored-value directions of this ill-conditioned system
        hh = h if step is None else step
        return (8.0 * diff(*point(hh), *point(-hh)) - diff(*point(2 * hh), *point(-2 * hh))) / (12.0 * hh)

    gen = torch.Generator(device="cuda").manual_seed(5)
    h = 1e-6
    # coefficient directions: step 1e-5.  Their derivative is a sum of
    # element terms that cancels to ~0.2% of its absolute sum, so at 1e-6 the
    # rounding of the perturbed solves is ~1e-5 of the signal (measured 1.2e-5
    # on one of ten directions); at 1e-5 it is ten times smaller, while the
    # stencil's O(h^4) truncation stays far below it
    hc = 1e-5
    errs = []
    v0 = vals.detach()
    b0 = b.detach()
    c0 = coef.detach()
    for t in range(32):
        # random relative perturbations: direction r * |theta|, r ~ N(0, I)
        if t < 11:
            d = torch.randn(b0.shape, generator=gen, device="cuda", dtype=torch.float64) * b0.abs()
            fd = derivative(lambda e: (v0, b0 + e * d))
            an = float(gb_ @ d)
            mag = float((gb_ * d).abs().sum())
        elif t < 22:
            d = torch.randn(v0.shape, generator=gen, device="cuda", dtype=torch.float64) * v0.abs()
            fd = derivative(lambda e: (v0 + e * d, b0))
            an = float(gv @ d)
            mag = float((gv * d).abs().sum())
        else:
            # a random smooth field over the element centroids (three cosine
            # modes of random wave vector, amplitude and phase) times c_e:
            # white-noise coefficient perturbations average out through the
            # elliptic operator (the derivative is ~1e-4 of sum |g_e d_e|) and
            # drown in the double-precision noise floor of the solves
            d = smooth_field(torch, g, gen) * c0
            with torch.no_grad():
                fd = derivative(lambda e: (asm(c0 + e * d), b0), hc)
            an = float(gc @ d)
            mag = float((gc * d).abs().sum())
        errs.append((abs(fd - an) / abs(fd), t, fd, an, abs(an) / mag))
    S.close()
    worst = sorted(errs, reverse=True)[:6]
    assert max(e[0] for e in errs) <= 1e-5, worst
