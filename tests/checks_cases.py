"""Small cases of every particle kernel, run by test_gpu_checks.py in a child process whose binding
loads the library named by BSPLINE_LIBRARY (the BSPLINE_CHECKS=1 build, or the default one).

Writes every output to the .npz file named on the command line, and the status code each plan (or
batch) reported after its calls; the parent compares the two builds' outputs bit for bit and checks
that no index check failed.  Held to the oracle here as well."""
import math
import sys

import numpy as np
import torch

from oracle import bspline_oracle as O
from paper_1201_4060_gb300 import bspline as B
from paper_1201_4060_gb300 import synth

TOL = {"f64": (1e-12, 1e-12), "f32": (2e-5, 5e-5), "bf16": (2e-2, 5e-2)}


def normwise(a, b):
    a = np.asarray(a, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def main(path):
    out, status = {}, {}
    for name, N, order, dtype, P, split in [("f32_o4", 32, 4, "f32", 20000, 0), ("f32_o6_split", 64, 6, "f32", 3000, 32),
                                            ("f64_o4", 16, 4, "f64", 3000, 0), ("bf16_o8", 32, 8, "bf16", 8000, 0),
                                            ("f32_o3", 16, 3, "f32", 5000, 0)]:
        half = synth.kolmogorov_field(N, seed=N + order).dense()
        xs = synth.clustered_particles(P, seed=order)
        plan = B.Plan(N, order, dtype)
        plan.set_gather_split(split)
        coef = plan.coeffs(torch.from_numpy(half).to(plan.uhat_dtype).cuda())
        x = torch.from_numpy(xs).cuda()
        u, g = plan.interp(coef, x)
        status[name] = B.bspline_status(plan.handle)[0]
        ref = half if dtype == "f64" else half.astype(np.complex64).astype(np.complex128)
        ru, rg = O.interpolate(ref, xs, order)
        tu, tg = TOL[dtype]
        assert normwise(u.cpu().numpy(), ru) < tu and normwise(g.cpu().numpy(), rg) < tg, name
        out[f"{name}_u"], out[f"{name}_g"] = u.cpu().numpy(), g.cpu().numpy()
        # sorted input, then the adjoint (spread, transposed transform, position gradient)
        perm = plan.sort_order(x).long()
        xp = x[perm].contiguous()
        us, gs = plan.interp(coef, xp, sorted=True)
        status[name + "_sorted"] = B.bspline_status(plan.handle)[0]
        assert torch.equal(us, u[perm]) and torch.equal(gs, g[perm]), name
        gu = torch.ones((P, 3), dtype=plan.out_dtype, device="cuda")
        gg = torch.full((P, 3, 3), 0.5, dtype=plan.out_dtype, device="cuda")
        gh, gx, gc = plan.spread_adjoint(x, gu, gg, coef=coef)
        status[name + "_adjoint"] = B.bspline_status(plan.handle)[0]
        out[f"{name}_gx"] = gx.cpu().numpy()
        if dtype != "f64":
            plan.set_deterministic(True)
            gh, gx, gc = plan.spread_adjoint(x, gu, gg, coef=coef)
            status[name + "_det"] = B.bspline_status(plan.handle)[0]
            out[f"{name}_gcoef_det"] = gc.cpu().numpy()
        plan.close()
    # a small batch through the persistent queue
    spec = [dict(N=16, seed=1, P=700), dict(N=48, seed=2, P=5000), dict(N=32, seed=3, P=0)]
    plans, uh, co, xsb, ou, og = [], [], [], [], [], []
    for f in spec:
        p = B.Plan(f["N"], 4, "f32")
        plans.append(p)
        uh.append(torch.from_numpy(synth.kolmogorov_field(f["N"], seed=f["seed"]).dense()).to(p.uhat_dtype).cuda())
        co.append(p.empty_coeffs())
        xsb.append(torch.from_numpy(synth.uniform_particles(f["P"], seed=f["seed"])).cuda())
        ou.append(torch.empty((f["P"], 3), device="cuda"))
        og.append(torch.empty((f["P"], 3, 3), device="cuda"))
    batch = B.Batch(plans)
    batch.capture(uh, co, xsb, ou, og, streams=2)
    batch.launch()
    status["batch"] = batch.status()[0]
    for i in range(2):
        out[f"batch{i}_u"], out[f"batch{i}_g"] = ou[i].cpu().numpy(), og[i].cpu().numpy()
    batch.close()
    # the allocation-free entry point
    N, order = 32, 4
    plan = B.Plan(N, order, "f32")
    coef = plan.coeffs(torch.from_numpy(synth.kolmogorov_field(N, seed=5).dense()).to(plan.uhat_dtype).cuda())
    x = torch.from_numpy(synth.uniform_particles(4000, seed=6)).cuda()
    u = torch.empty((4000, 3), device="cuda")
    g = torch.empty((4000, 3, 3), device="cuda")
    rc = B.bspline_interp_noalloc(coef.data_ptr(), N, order, B.F32, 2.0 * math.pi, x.data_ptr(), 4000, u.data_ptr(),
                                  g.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    assert rc == B.OK
    torch.cuda.synchronize()
    out["noalloc_u"], out["noalloc_g"] = u.cpu().numpy(), g.cpu().numpy()
    plan.close()
    np.savez(path, **out, **{f"status_{k}": np.array(v) for k, v in status.items()})


if __name__ == "__main__":
    main(sys.argv[1])
