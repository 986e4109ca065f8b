"""A seeded sweep of randomly drawn configurations of the whole path against the oracle.

Each case draws a grid size (radix-2 and radix-3 grids), an order 2..8, a coefficient type, a domain length,
a prefilter, a gather split (all bricks staged, the automatic split, or every brick by the direct gather),
gradients on or off, and a particle set that mixes uniform positions over three periods (so the periodic
wrap is exercised on both sides), Gaussian clumps (bricks split into several work items), positions exactly
on grid nodes and on the period's ends, and a ragged count.  Some cases pass the particles in the plan's brick
order with BSPLINE_INTERP_SORTED.  The GPU result is compared with the oracle element by element under the
tolerances of the parity tests (FP64 1e-12; FP32 and BF16 as derived there).  A second sweep does the same
for the adjoint (bspline_spread_adjoint against the oracle's spread, transposed transform and position
gradient).
"""

import numpy as np
import pytest

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import synth

torch = pytest.importorskip("torch")

TOL = {"f64": (1e-12, 1e-12), "f32": (2e-5, 5e-5), "bf16": (2e-2, 5e-2)}
GRIDS = [8, 16, 32, 48, 64, 96]
CASES = 24


@pytest.fixture(scope="module")
def B():
    from paper_1201_4060_gb300 import _build
    _build.build()
    from paper_1201_4060_gb300 import bspline
    assert torch.cuda.is_available()
    return bspline


def normwise(a, b):
    """max |a - b| / max |b|, complex values compared as complex."""
    a = np.asarray(a)
    b = np.asarray(b)
    a = a.astype(np.complex128) if np.iscomplexobj(a) or np.iscomplexobj(b) else a.astype(np.float64)
    b = b.astype(a.dtype)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def draw_case(i):
    rng = np.random.default_rng(9000 + i)
    N = int(rng.choice(GRIDS))
    order = int(rng.integers(2, 9))
    dtype = ["f64", "f32", "bf16"][i % 3]
    L = float(rng.uniform(0.5, 12.0))
    prefilter = "l2" if (dtype == "f64" and rng.random() < 0.4) else "interp"
    split = [0, None, 1 << 30][int(rng.integers(0, 3))] if dtype != "f64" else None
    grad = bool(rng.random() < 0.8)
    presorted = bool(dtype != "bf16" and rng.random() < 0.3)
    P = int(rng.integers(1, 6000))
    h = L / N
    parts = [rng.uniform(-L, 2 * L, size=(P, 3))]
    if P > 20:
        nc = int(rng.integers(1, 4))
        centres = rng.uniform(0, L, size=(nc, 3))
        clump = centres[rng.integers(0, nc, size=P // 2)] + 0.3 * h * rng.standard_normal((P // 2, 3))
        parts.append(clump)
    nodes = rng.integers(-N, 2 * N, size=(17, 3)) * h                  # exactly on nodes
    ends = np.array([[0.0, L, 0.5 * L], [L, L, L], [-0.0, 0.0, L - 1e-15], [np.nextafter(L, 0.0), 0.0, 0.0]])
    x = np.concatenate(parts + [nodes, ends])[rng.permutation(sum(len(p) for p in parts) + len(nodes) + len(ends))]
    return dict(N=N, order=order, dtype=dtype, L=L, prefilter=prefilter, split=split, grad=grad,
                presorted=presorted, seed=int(rng.integers(1 << 30)), x=np.ascontiguousarray(x))


@pytest.mark.gpu
@pytest.mark.parametrize("i", range(CASES))
def test_random_configuration_matches_oracle(B, i):
    c = draw_case(i)
    N, order, dtype, L = c["N"], c["order"], c["dtype"], c["L"]
    half = synth.kolmogorov_field(N, seed=c["seed"]).dense()
    plan = B.Plan(N, order, dtype, L=L, prefilter=c["prefilter"])
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    if c["split"] is not None:
        plan.set_gather_split(c["split"])
    xs = c["x"]
    x = torch.from_numpy(xs).cuda()
    if c["presorted"]:
        perm = plan.sort_order(x).long()
        xin = x[perm].contiguous()
    else:
        perm = None
        xin = x
    res = plan.interp(coef, xin, grad=c["grad"], sorted=c["presorted"])
    u, g = res if c["grad"] else (res, None)
    if perm is not None:                                   # back to the drawn order
        inv = torch.empty_like(perm)
        inv[perm] = torch.arange(len(perm), device=perm.device)
        u = u[inv]
        g = g[inv] if g is not None else None
    torch.cuda.synchronize()
    assert plan.status() == 0, c
    src = half if dtype == "f64" else half.astype(np.complex64).astype(np.complex128)
    ru, rg = O.interpolate(src, xs, order, L=L, kind=c["prefilter"])
    tu, tg = TOL[dtype]
    eu = normwise(u.double().cpu().numpy(), ru)
    assert eu < tu, (c["N"], order, dtype, L, c["prefilter"], c["split"], c["presorted"], eu)
    if g is not None:
        eg = normwise(g.double().cpu().numpy(), rg)
        assert eg < tg, (c["N"], order, dtype, L, c["prefilter"], c["split"], c["presorted"], eg)
    plan.close()


def test_sweep_draws_cover_the_options():
    """The drawn cases reach every type, both prefilters, every gather split, the sorted flag, the
    no-gradient form, radix-3 grids and orders at both ends (checked on the CPU, no GPU needed)."""
    cs = [draw_case(i) for i in range(CASES)]
    assert {c["dtype"] for c in cs} == {"f64", "f32", "bf16"}
    assert {c["prefilter"] for c in cs} == {"interp", "l2"}
    assert {c["split"] for c in cs if c["dtype"] != "f64"} >= {0, None, 1 << 30}
    assert any(c["presorted"] for c in cs) and any(not c["grad"] for c in cs)
    assert any(c["N"] % 3 == 0 for c in cs)
    assert min(c["order"] for c in cs) <= 3 and max(c["order"] for c in cs) >= 7


# ----------------------------------------------------------------------- the adjoint

ADJ_CASES = 12
TOL_ADJ = {"f64": (1e-12, 1e-12, 1e-12), "f32": (1e-5, 2e-5, 2e-4)}    # spread, transposed transform, g_x


def draw_adjoint_case(i):
    rng = np.random.default_rng(9500 + i)
    N = int(rng.choice(GRIDS[:5]))
    order = int(rng.integers(2, 9))
    dtype = "f64" if i % 2 == 0 else "f32"
    L = float(rng.uniform(0.5, 12.0))
    P = int(rng.integers(1, 4000))
    x = rng.uniform(-L, 2 * L, size=(P, 3))
    x[: min(P, 5)] = rng.integers(-N, 2 * N, size=(min(P, 5), 3)) * (L / N)      # on nodes
    return dict(N=N, order=order, dtype=dtype, L=L, x=np.ascontiguousarray(x),
                prefilter="l2" if rng.random() < 0.3 else "interp", grad=bool(rng.random() < 0.75),
                det=bool(dtype == "f32" and rng.random() < 0.5), seed=int(rng.integers(1 << 30)))


@pytest.mark.gpu
@pytest.mark.parametrize("i", range(ADJ_CASES))
def test_random_adjoint_configuration_matches_oracle(B, i):
    """bspline_spread_adjoint against oracle.spread, oracle.adjoint_transform and
    oracle.position_gradient on randomly drawn grids, orders, lengths, prefilters, cotangents with and
    without the gradient part, and the deterministic spread."""
    c = draw_adjoint_case(i)
    N, order, dtype, L, xs = c["N"], c["order"], c["dtype"], c["L"], c["x"]
    P = len(xs)
    plan = B.Plan(N, order, dtype, L=L, prefilter=c["prefilter"])
    if c["det"]:
        plan.set_deterministic(True)
    half = synth.kolmogorov_field(N, seed=c["seed"]).dense()
    coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
    rng = np.random.default_rng(c["seed"])
    gu_t = torch.from_numpy(rng.standard_normal((P, 3))).to(plan.out_dtype).cuda()
    gg_t = torch.from_numpy(rng.standard_normal((P, 3, 3))).to(plan.out_dtype).cuda() if c["grad"] else None
    gh, gx, gc = plan.spread_adjoint(torch.from_numpy(xs).cuda(), gu_t, gg_t, coef=coef)
    torch.cuda.synchronize()
    assert plan.status() == 0, c
    gu = gu_t.double().cpu().numpy()
    gg = gg_t.double().cpu().numpy() if gg_t is not None else None
    rc = O.spread(xs, gu, gg, N, order, L=L)
    ts, tf, tx = TOL_ADJ[dtype]
    assert normwise(gc.double().cpu().numpy(), rc) < ts, c["N"]
    assert normwise(gh.cpu().numpy(), O.adjoint_transform(rc, order, c["prefilter"])) < tf, c["N"]
    src = half if dtype == "f64" else half.astype(np.complex64).astype(np.complex128)
    rx = O.position_gradient(O.coefficients(src, order, c["prefilter"]), xs, gu, gg, order, L=L)
    assert normwise(gx.cpu().numpy(), rx) < tx, c["N"]
    plan.close()


def test_adjoint_sweep_draws_cover_the_options():
    cs = [draw_adjoint_case(i) for i in range(ADJ_CASES)]
    assert {c["dtype"] for c in cs} == {"f64", "f32"}
    assert {c["prefilter"] for c in cs} == {"interp", "l2"}
    assert any(c["det"] for c in cs) and any(not c["grad"] for c in cs)
    assert any(c["N"] % 3 == 0 for c in cs)
