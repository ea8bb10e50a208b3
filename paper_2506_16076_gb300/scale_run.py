"""Scale run: a long batched forward run followed by the checkpointed discrete adjoint
over its last steps, on one GPU.

    python -m paper_2506_16076_gb300.scale_run --workload cyl_m25_4096 --forward 200 \
        --adjoint 100 --checkpoint-every 10

The first (forward - adjoint) steps run plainly; the last `adjoint` steps keep a state
checkpoint every K steps and no per-step viscosity (the backward run recomputes it from
the replayed states). J is the wall-drag functional after the last step; the adjoint
carries dJ/de back to the start of the differentiated window. Prints one JSON line with
the forward and adjoint rates and the device memory in use.
"""
import argparse
import json
import time

import torch

from . import adjoint as ADJ
from . import fcsdnn
from . import workloads as W


def device_used_gb():
    free, total = torch.cuda.mem_get_info()
    return (total - free) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cyl_m25_4096")
    ap.add_argument("--forward", type=int, default=200)
    ap.add_argument("--adjoint", type=int, default=100)
    ap.add_argument("--checkpoint-every", type=int, default=10)
    a = ap.parse_args()
    w = W.WORKLOADS[a.workload]()
    t0 = time.time()
    ctx = fcsdnn.Context(w)
    init_s = time.time() - t0
    e = torch.from_numpy(W.flatten(W.initial_state(w))).cuda()
    nplain = a.forward - a.adjoint
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.empty(ctx.P, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t1 = time.time()
    for n in range(nplain):
        ctx.rk_step(e, dt, mu, fcsdnn.STEP_FILTER if n >= 1 else 0)
    torch.cuda.synchronize()
    t2 = time.time()
    del mu
    # the differentiated window: filter on every step (all n >= 1 of the run)
    eN, tr = ADJ.forward(ctx, e, a.adjoint, a.checkpoint_every, filter=True, store_mu=False,
                         first_filtered=0 if nplain >= 1 else 1)
    torch.cuda.synchronize()
    t3 = time.time()
    J, dJde = ADJ.drag(ctx, eN)
    lam0, gbc = ADJ.backward(ctx, tr, dJde)
    torch.cuda.synchronize()
    t4 = time.time()
    status = ctx.sync_status(eN)
    out = {
        "workload": a.workload, "points": ctx.P, "active_points": ctx.active, "patches": len(w.patches),
        "init_s": round(init_s, 2), "forward_steps": a.forward, "adjoint_steps": a.adjoint,
        "checkpoint_every": a.checkpoint_every,
        "forward_ms_per_step": 1e3 * (t3 - t1) / a.forward,
        "forward_point_updates_per_s": 5 * ctx.active * a.forward / (t3 - t1),
        "adjoint_ms_per_step": 1e3 * (t4 - t3) / a.adjoint,
        "adjoint_forward_ratio": ((t4 - t3) / a.adjoint) / ((t3 - t1) / a.forward),
        "J": J.item(), "lambda_finite": bool(torch.isfinite(lam0).all()), "state_status": int(status),
        "device_memory_in_use_gb": round(device_used_gb(), 1),
        "torch_peak_gb": round(torch.cuda.max_memory_allocated() / 1e9, 1),
        "note": "wall-clock with host synchronisation only at the phase ends; forward includes checkpoint copies",
    }
    _ = t2
    print(json.dumps(out))


if __name__ == "__main__":
    main()
