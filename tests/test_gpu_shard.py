"""Sharded execution (fc_shard) on one GPU: two or three ranks emulated as contexts of one
process, one host thread each, exchanging through the in-process transport. After a few
time steps of Algorithm 1 (projection with the inter-patch exchange, viscosity with the
cross-patch blending, per-step filter, time step of eq. CFL, five SSPRK stages) every
rank's owned patches equal the unsharded context's result bit for bit (the unsharded
step's parity with the oracle is covered by the parity tests), and so does the
checkpointed adjoint with the exchange reversed between ranks."""
import threading

import pytest
import torch

from paper_2506_16076_gb300 import shard, workloads as W
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

NSTEPS = 4


def _run_unsharded(gpu_lib, w, st0):
    ctx = gpu_lib.Context(w)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        e = to_dev(st0)
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        mu = torch.zeros(e.shape[1], dtype=torch.float64, device="cuda")
        dts = []
        for n in range(NSTEPS):
            ctx.rk_step(e, dt, mu, gpu_lib.STEP_FILTER if n else 0)
            dts.append(dt.clone())
    s.synchronize()
    return e.cpu(), mu.cpu(), [d.item() for d in dts]


def _run_sharded(gpu_lib, w, st0, owner, nranks):
    hub = shard.LocalHub(nranks)
    ctxs = [gpu_lib.Context(w) for _ in range(nranks)]
    for r, c in enumerate(ctxs):
        c.shard(nranks, r, owner, shard.LocalComm(hub, r))
    out, errs = [None] * nranks, []

    def rank_main(r):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                e = to_dev(st0)
                dt = torch.zeros(1, dtype=torch.float64, device="cuda")
                mu = torch.zeros(e.shape[1], dtype=torch.float64, device="cuda")
                dts = []
                for n in range(NSTEPS):
                    ctxs[r].rk_step(e, dt, mu, gpu_lib.STEP_FILTER if n else 0)
                    dts.append(dt.clone())
            s.synchronize()
            out[r] = (e.cpu(), mu.cpu(), [d.item() for d in dts])
        except Exception as ex:  # reported by the main thread
            errs.append((r, ex))
            hub.barrier.abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(nranks)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return ctxs, out


def _wall_form(w):
    import dataclasses
    return dataclasses.replace(w, params=dataclasses.replace(w.params, wall_form=1))


@pytest.mark.parametrize("name,nranks", [("multi", 2), ("multi_adiabatic", 3), ("grid_curved", 2),
                                         ("grid_curved_product_wall", 2)])
def test_sharded_steps_equal_unsharded(gpu_lib, name, nranks):
    w = {"multi": W.small_multipatch, "multi_adiabatic": lambda: W.small_multipatch(W.ADIABATIC),
         "grid_curved": W.small_multipatch_grid,
         "grid_curved_product_wall": lambda: _wall_form(W.small_multipatch_grid())}[name]()
    st0 = W.random_smooth_state(w, seed=21, amp=0.05)
    owner = shard.partition(w, nranks)
    assert sorted(set(owner)) == list(range(nranks))
    e_ref, mu_ref, dts_ref = _run_unsharded(gpu_lib, w, st0)
    ctxs, out = _run_sharded(gpu_lib, w, st0, owner, nranks)
    offs = w.offsets
    for r in range(nranks):
        e, mu, dts = out[r]
        assert dts == dts_ref  # the global minimum of eq. CFL on every rank
        for p, o in enumerate(owner):
            if o != r:
                continue
            sl = slice(offs[p], offs[p + 1])
            assert torch.equal(e[:, sl], e_ref[:, sl]), (r, p)
            assert torch.equal(mu[sl], mu_ref[sl]), (r, p)
    # the exchange plans of the ranks agree pairwise
    for a in range(nranks):
        for b in range(nranks):
            if a != b:
                for which in (0, 1):
                    assert ctxs[a].shard_counts(which, b)[0] == ctxs[b].shard_counts(which, a)[1]


def _mach2_small():
    import dataclasses
    import math
    w = W.small_multipatch(W.ADIABATIC)
    a = math.radians(2.0)
    fs = (1.4, 2.0 * math.cos(a), 2.0 * math.sin(a), 1.0)
    return W.Workload("small_m2", [dataclasses.replace(p, bc=(fs,) * 4) for p in w.patches], w.params, fs,
                      "freestream", 4)


def test_sharded_drag_gradients_equal_unsharded(gpu_lib):
    # the checkpointed adjoint (fc_adjoint_step, the exchange reversed between ranks) and
    # the parameter gradients: owned lambda_0 and dJ/drho_0 bit for bit, J and dJ/d(M, alpha)
    # as the sum of the ranks' parts (their order of summation differs)
    from paper_2506_16076_gb300 import adjoint as ADJ
    w = _mach2_small()
    nsteps, K, nranks = 4, 2, 2
    ctx = gpu_lib.Context(w)
    e0 = to_dev(W.initial_state(w))
    J, dM, dA, drho, _ = ADJ.drag_gradients(w, ctx, e0, nsteps, K, filter=True)
    owner = shard.partition(w, nranks)
    hub = shard.LocalHub(nranks)
    ctxs = [gpu_lib.Context(w) for _ in range(nranks)]
    for r, c in enumerate(ctxs):
        c.shard(nranks, r, owner, shard.LocalComm(hub, r))
    out, errs = [None] * nranks, []

    def rank_main(r):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                out[r] = ADJ.drag_gradients(w, ctxs[r], to_dev(W.initial_state(w)), nsteps, K, filter=True)
            s.synchronize()
        except Exception as ex:  # reported by the main thread
            errs.append((r, ex))
            hub.barrier.abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(nranks)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    assert abs(sum(o[0] for o in out) - J) <= 1e-14 * abs(J)
    for k, ref in ((1, dM), (2, dA)):
        got = sum(o[k] for o in out)
        assert abs(got - ref) <= 1e-12 * max(abs(ref), 1e-300), (k, got, ref)
    offs = w.offsets
    for r in range(nranks):
        for p, o in enumerate(owner):
            if o == r:
                sl = slice(offs[p], offs[p + 1])
                assert torch.equal(out[r][3][sl].cpu(), drho[sl].cpu()), (r, p)


def test_sharded_context_refuses_graph_and_tuning(gpu_lib):
    w = W.small_multipatch()
    owner = shard.partition(w, 2)
    hub = shard.LocalHub(1)
    ctx = gpu_lib.Context(w)
    ctx.shard(2, 0, owner, shard.LocalComm(hub, 0))
    e = to_dev(W.initial_state(w))
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.zeros(e.shape[1], dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.FcError):
        ctx.rk_step(e, dt, mu, gpu_lib.STEP_GRAPH)
    with pytest.raises(gpu_lib.FcError):
        ctx.rk_step(e, dt, mu, gpu_lib.STEP_PER_PATCH)
    with pytest.raises(gpu_lib.FcError):
        ctx.autotune()
    with pytest.raises(gpu_lib.FcError):
        ctx.shard(2, 0, owner, shard.LocalComm(hub, 0))
