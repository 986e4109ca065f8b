"""Batches of independent fields replayed as one CUDA graph (bspline_batch_*).

The graph runs the same kernels on the same inputs as the single-field calls,
so its outputs must equal theirs bit for bit (the forward path has no
atomics); one field per grid size is also held to the oracle.
"""
import math

import numpy as np
import pytest

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 2.0 * math.pi
TOL32 = {"u": 2e-5, "grad": 5e-5}


@pytest.fixture(scope="module")
def B():
    from paper_1201_4060_gb300 import _build
    _build.build()
    from paper_1201_4060_gb300 import bspline
    assert torch.cuda.is_available()
    return bspline


def normwise(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _fields(B, spec, dtype="f32", order=4):
    plans, uh, co, xs, ou, og, halves, xnp = [], [], [], [], [], [], [], []
    shared = {}
    for f in spec:
        key = f.get("share")
        if key is not None and key in shared:
            plan = shared[key]
        else:
            plan = B.Plan(f["N"], order, dtype)
            if key is not None:
                shared[key] = plan
        half = synth.kolmogorov_field(f["N"], seed=f["field_seed"]).dense()
        x = synth.uniform_particles(f["P"], seed=f["particle_seed"])
        plans.append(plan)
        halves.append(half)
        xnp.append(x)
        uh.append(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
        co.append(plan.empty_coeffs())
        xs.append(torch.from_numpy(x).cuda())
        ou.append(torch.full((f["P"], 3), float("nan"), dtype=plan.out_dtype, device="cuda"))
        og.append(torch.full((f["P"], 3, 3), float("nan"), dtype=plan.out_dtype, device="cuda"))
    return plans, uh, co, xs, ou, og, halves, xnp


SPEC = [dict(N=16, field_seed=1, particle_seed=11, P=700),
        dict(N=48, field_seed=2, particle_seed=12, P=5000),
        dict(N=32, field_seed=3, particle_seed=13, P=1, share="a"),
        dict(N=32, field_seed=4, particle_seed=14, P=20000, share="a"),   # same plan as the previous field
        dict(N=96, field_seed=5, particle_seed=15, P=3000),
        dict(N=64, field_seed=6, particle_seed=16, P=0),
        dict(N=192, field_seed=7, particle_seed=17, P=12000)]


@pytest.mark.parametrize("streams", [1, 3])
def test_batch_graph_equals_single_field_calls(B, streams):
    plans, uh, co, xs, ou, og, halves, xnp = _fields(B, SPEC)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=streams)
    batch.launch()
    torch.cuda.synchronize()
    for i, f in enumerate(SPEC):
        c = plans[i].coeffs(uh[i])
        if f["P"] == 0:
            assert torch.equal(c, co[i])
            continue
        u, g = plans[i].interp(c, xs[i])
        torch.cuda.synchronize()
        assert torch.equal(c, co[i])
        assert torch.equal(u, ou[i]) and torch.equal(g, og[i])
    # one field of each grid size against the oracle
    for i in (1, 3, 4, 6):
        ru, rg = O.interpolate(halves[i].astype(np.complex64).astype(np.complex128), xnp[i], 4)
        assert normwise(ou[i].cpu().numpy(), ru) < TOL32["u"]
        assert normwise(og[i].cpu().numpy(), rg) < TOL32["grad"]
    batch.close()


def test_batch_relaunch_and_autotune(B):
    plans, uh, co, xs, ou, og, _, _ = _fields(B, SPEC)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=2)
    batch.launch()
    torch.cuda.synchronize()
    ref_u = [t.clone() for t in ou]
    ref_g = [t.clone() for t in og]
    for t in ou + og:
        t.fill_(float("nan"))
    k, ms = batch.autotune()
    assert 1 <= k <= 16 and ms > 0
    for t in ou + og:
        t.fill_(float("nan"))
    batch.launch()
    batch.launch()
    torch.cuda.synchronize()
    for i in range(len(SPEC)):
        assert torch.equal(ou[i], ref_u[i]) and torch.equal(og[i], ref_g[i])
        assert plans[i].status() == 0
    batch.close()


def test_batch_u_only_and_f64(B):
    spec = SPEC[:3]
    plans, uh, co, xs, ou, og, halves, xnp = _fields(B, spec, dtype="f64", order=6)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, None, streams=2)           # u only
    batch.launch()
    torch.cuda.synchronize()
    for i in range(len(spec)):
        ru, _ = O.interpolate(halves[i], xnp[i], 6)
        assert normwise(ou[i].cpu().numpy(), ru) < 1e-12
        assert torch.isnan(og[i]).all()                      # untouched
    batch.close()


def test_batch_rejects_bad_arguments(B):
    plans, uh, co, xs, ou, og, _, _ = _fields(B, SPEC[:2])
    batch = B.Batch(plans)
    lib = B.lib()
    assert lib.bspline_batch_launch(batch.handle, None) == B.ERR_INVALID_ARG          # not captured
    assert lib.bspline_batch_autotune(batch.handle, None, None, None) == B.ERR_INVALID_ARG
    with pytest.raises(B.BSplineError):
        batch.capture(uh, co, xs, ou, og, streams=0)
    co_bad = [co[0], uh[1]]                                  # coefficients aliasing u_hat
    with pytest.raises(B.BSplineError):
        batch.capture(uh, co_bad, xs, ou, og, streams=1)
    batch.close()


def _single_field(plans, uh, xs, i):
    c = plans[i].coeffs(uh[i])
    u, g = plans[i].interp(c, xs[i])
    torch.cuda.synchronize()
    return c, u, g


@pytest.mark.parametrize("by,item", [(12, 2048), (8, 512), (16, 1024)])
def test_batch_queue_layouts_equal_single_field_calls(B, by, item):
    """The persistent queue kernel (every field's count, scan, placement and gather tasks in one launch)
    gives the single-field calls' bits at every brick y extent and item size."""
    plans, uh, co, xs, ou, og, halves, xnp = _fields(B, SPEC)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=2)
    batch.set_layout(queue=1, brick_y=by, item_particles=item)
    cfg = batch.config()
    assert cfg["queue"] == 1 and cfg["brick_y"] == by and cfg["item_particles"] == item
    # two transform kernels per grid size (the fields of one size in one launch each) and the one queue kernel
    assert cfg["kernel_nodes"] == 2 * len({f["N"] for f in SPEC}) + 1
    batch.launch()
    assert batch.status() == (B.OK, 0)
    for i, f in enumerate(SPEC):
        c, u, g = _single_field(plans, uh, xs, i)
        assert torch.equal(c, co[i])
        if f["P"]:
            assert torch.equal(u, ou[i]) and torch.equal(g, og[i]), (i, by, item)
    ru, rg = O.interpolate(halves[6].astype(np.complex64).astype(np.complex128), xnp[6], 4)
    assert normwise(ou[6].cpu().numpy(), ru) < TOL32["u"] and normwise(og[6].cpu().numpy(), rg) < TOL32["grad"]
    batch.close()


def test_batch_queue_wait_timeout_and_next_launch(B):
    """A queue entry left unpublished (the first count task of field 0 skips its signal): the scan of field
    0 waits until its bounded wait runs out, the launch ends, bspline_batch_status reports TIMEOUT; the next
    launch without the hook is correct and reports OK."""
    plans, uh, co, xs, ou, og, _, _ = _fields(B, SPEC)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=2)
    batch.set_layout(queue=1)
    batch.set_test_hooks(B.TEST_DROP_QUEUE_SIGNAL)
    batch.launch()
    rc, _ = batch.status()
    assert rc == B.ERR_TIMEOUT
    batch.set_test_hooks(0)
    for t in ou + og:
        t.fill_(float("nan"))
    batch.launch()
    assert batch.status() == (B.OK, 0)
    for i, f in enumerate(SPEC):
        if f["P"]:
            _, u, g = _single_field(plans, uh, xs, i)
            assert torch.equal(u, ou[i]) and torch.equal(g, og[i])
    batch.close()


def test_batch_queue_nonfinite_positions(B):
    spec = [dict(N=32, field_seed=21, particle_seed=31, P=3000), dict(N=48, field_seed=22, particle_seed=32, P=900)]
    plans, uh, co, xs, ou, og, _, _ = _fields(B, spec)
    xs[1][[5, 17]] = torch.tensor([[float("nan"), 0.0, 0.0], [1.0, float("inf"), 1.0]], dtype=torch.float64,
                                  device="cuda")
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=1)
    assert batch.config()["queue"] == 1
    batch.launch()
    assert batch.status() == (B.ERR_NONFINITE_INPUT, 2)
    assert torch.isnan(ou[1][[5, 17]]).all() and torch.isnan(og[1][[5, 17]]).all()
    _, u, g = _single_field(plans, uh, xs, 1)
    assert torch.equal(torch.isnan(u), torch.isnan(ou[1]))
    ok = ~torch.isnan(u[:, 0])
    assert torch.equal(u[ok], ou[1][ok]) and torch.equal(g[ok], og[1][ok])
    batch.close()


def test_batch_queue_only_where_fields_allow(B):
    """u only or FP64: the per-field graph; requiring the queue there is refused."""
    spec = SPEC[:2]
    plans, uh, co, xs, ou, og, _, _ = _fields(B, spec, dtype="f64", order=4)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=1)
    assert batch.config()["queue"] == 0
    with pytest.raises(B.BSplineError) as exc:
        batch.set_layout(queue=1)
    assert exc.value.code == B.ERR_NOT_IMPLEMENTED
    batch.close()
    plans, uh, co, xs, ou, og, _, _ = _fields(B, spec)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, None, streams=1)            # u only
    assert batch.config()["queue"] == 0
    batch.close()


def test_batch_queue_autotune_and_its_cache(B, tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("BSPLINE_AUTOTUNE_CACHE", str(cache))
    plans, uh, co, xs, ou, og, _, _ = _fields(B, SPEC)
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=1)
    k, ms = batch.autotune()
    cfg = batch.config()
    assert ms > 0 and cfg["queue"] == 1 and cfg["brick_y"] in (8, 12, 16) and cfg["item_particles"] in (512, 1024,
                                                                                                          2048)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and '"brick_y"' in lines[0]
    batch.launch()
    assert batch.status() == (B.OK, 0)
    ref = [t.clone() for t in ou]
    batch.close()
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=1)
    k2, ms2 = batch.autotune()                                # from the cache: no timing
    assert ms2 == 0.0 and k2 == k and batch.config()["brick_y"] == cfg["brick_y"]
    batch.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(ref, ou))
    batch.close()


def test_batch_band_limited_fields_equal_single_field_calls(B):
    """Plans told that their fields are band-limited (bspline_plan_set_band, K = N/3 here and K = N/4 for a
    second plan of one grid size: two transform groups of that size) run their transforms on the band in
    the batch as in single-field calls: the same bits, and the full path's bits too."""
    spec = [dict(N=48, field_seed=41, particle_seed=51, P=4000, K=16), dict(N=64, field_seed=42, particle_seed=52,
            P=9000, K=21), dict(N=64, field_seed=43, particle_seed=53, P=3000, K=16)]
    plans, uh, co, xs, ou, og = [], [], [], [], [], []
    for f in spec:
        plan = B.Plan(f["N"], 4, "f32")
        plan.set_band(f["K"])
        half = synth.kolmogorov_field(f["N"], seed=f["field_seed"], kmax=f["K"]).dense()
        plans.append(plan)
        uh.append(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
        co.append(plan.empty_coeffs())
        xs.append(torch.from_numpy(synth.uniform_particles(f["P"], seed=f["particle_seed"])).cuda())
        ou.append(torch.empty((f["P"], 3), dtype=torch.float32, device="cuda"))
        og.append(torch.empty((f["P"], 3, 3), dtype=torch.float32, device="cuda"))
    batch = B.Batch(plans)
    batch.capture(uh, co, xs, ou, og, streams=2)
    batch.launch()
    assert batch.status() == (B.OK, 0)
    for i, f in enumerate(spec):
        c, u, g = _single_field(plans, uh, xs, i)
        full = B.Plan(f["N"], 4, "f32")
        cf = full.coeffs(uh[i])
        torch.cuda.synchronize()
        assert torch.equal(c, co[i]) and torch.equal(cf, co[i])
        assert torch.equal(u, ou[i]) and torch.equal(g, og[i])
    batch.close()
