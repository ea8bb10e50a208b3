"""The sharded time step on CPU ranks (gloo, world size 2): each rank owns the patches
fc_partition gives it and advances only those, with the oracle's operator; the fringe
values a rank owes to the other (interpolated from its donors), the window sums of the
cross-patch blending and the time step's minimum travel through the same transport the
GPU path uses (shard.DistComm), in the library's message layout (per peer blocks, in the
order of the unsharded receiver list). After the steps every rank's owned patches equal
the single-domain oracle's bit for bit (Algorithm 1, the communication step)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

NSTEPS = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class ShardedOracle:
    """The oracle's step of one rank: owned patches only, the couplings through comm."""

    def __init__(self, w, owner, rank, comm):
        from oracle import solver as S
        self.sv = S.Solver(w)
        self.owner, self.rank, self.comm = owner, rank, comm
        self.n = max(owner) + 1
        it = self.sv.conn.items
        # fringe receivers (p, k) per peer: those this rank interpolates for q, and those it gets
        self.fsend = [[(p, k) for p in range(len(it)) for k in range(len(it[p]["j"]))
                       if owner[p] == q and it[p]["donor"][k] >= 0 and owner[it[p]["donor"][k]] == rank]
                      if q != rank else [] for q in range(self.n)]
        self.frecv = [[(p, k) for p in range(len(it)) for k in range(len(it[p]["j"]))
                       if owner[p] == rank and it[p]["donor"][k] >= 0 and owner[it[p]["donor"][k]] == q]
                      if q != rank else [] for q in range(self.n)]
        # cross-patch window sums per peer: (p, entry) with owner[p] = dst rank, owner[q] = src rank
        cr = self.sv.sb.cross
        self.vsend = [[(p, e) for p in range(len(cr)) for e in range(len(cr[p]))
                       if owner[p] == q and owner[cr[p][e][0]] == rank] if q != rank else []
                      for q in range(self.n)]
        self.vrecv = [[(p, e) for p in range(len(cr)) for e in range(len(cr[p]))
                       if owner[p] == rank and owner[cr[p][e][0]] == q] if q != rank else []
                      for q in range(self.n)]

    def _exchange(self, blocks_send, sizes_recv):
        send = torch.from_numpy(np.concatenate([b.ravel() for b in blocks_send] + [np.zeros(0)]))
        sc = [b.size for b in blocks_send]
        recv = torch.empty(sum(sizes_recv), dtype=torch.float64)
        self.comm.exchange(send, sc, recv, sizes_recv)
        out, off = [], 0
        for k in sizes_recv:
            out.append(recv[off:off + k].numpy())
            off += k
        return out

    def project(self, states):
        sv, it = self.sv, self.sv.conn.items
        sv.apply_bc(states)
        sv.conn.exchange(states)  # right for receivers whose donors are this rank's
        blocks = [np.array([states[p][:, it[p]["j"][k], it[p]["i"][k]] for (p, k) in lst]).reshape(-1)
                  for lst in self.fsend]
        got = self._exchange(blocks, [4 * len(lst) for lst in self.frecv])
        for q, lst in enumerate(self.frecv):
            vals = got[q].reshape(-1, 4)
            for m, (p, k) in enumerate(lst):
                states[p][:, it[p]["j"][k], it[p]["i"][k]] = vals[m]
        return states

    def viscosity(self, states):
        from oracle import viscosity as V
        sv, sb, cr = self.sv, self.sv.sb, self.sv.sb.cross
        muhat = [V.preliminary(g, e, sv.prm)[0] if self.owner[p] == self.rank else np.zeros_like(e[0])
                 for p, (g, e) in enumerate(zip(sv.geos, states))]
        num_own = [sb.window_sum(g, m) for g, m in zip(sv.geos, muhat)]
        blocks = [np.concatenate([num_own[cr[p][e][0]][cr[p][e][3], cr[p][e][4]] for (p, e) in lst] + [np.zeros(0)])
                  for lst in self.vsend]
        got = self._exchange(blocks, [sum(len(cr[p][e][1]) for (p, e) in lst) for lst in self.vrecv])
        remote = {}
        for q, lst in enumerate(self.vrecv):
            off = 0
            for (p, e) in lst:
                k = len(cr[p][e][1])
                remote[(p, e)] = got[q][off:off + k]
                off += k
        out = []
        for p, g in enumerate(sv.geos):
            if self.owner[p] != self.rank:
                out.append(np.zeros_like(num_own[p]))
                continue
            num = num_own[p].copy()
            for e, (q, jj, ii, z2, z1) in enumerate(cr[p]):
                num[jj, ii] += remote[(p, e)] if self.owner[q] != self.rank else num_own[q][z2, z1]
            den = sb.den[p]
            mu = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
            out.append(np.where(g.blank, 0.0, mu))
        return out

    def dt(self, states, mus):
        from oracle import euler
        sv, best = self.sv, np.inf
        for p, (g, e, m) in enumerate(zip(sv.geos, states, mus)):
            v = ~g.blank
            if self.owner[p] != self.rank or not v.any():
                continue
            S_ = euler.mwsb(e, sv.prm.gamma)[v].max()
            best = min(best, sv.prm.cfl / (S_ / g.htil + m[v].max() / g.htil ** 2))
        loc = torch.tensor([best / np.pi], dtype=torch.float64)
        out = torch.empty(1, dtype=torch.float64)
        self.comm.allmin(loc, out)
        return out.item()

    def step(self, states, n):
        from oracle.solver import SSP54_ALPHA, SSP54_BETA
        sv = self.sv
        states = [e.copy() for e in states]
        self.project(states)
        mu = self.viscosity(states)
        if n >= sv.filter_from_step:
            states = [sv.filter_patch(g, e) if self.owner[p] == self.rank else e
                      for p, (g, e) in enumerate(zip(sv.geos, states))]
            self.project(states)
        dt = self.dt(states, mu)
        u, Ls = [states], []
        for i in range(5):
            Ls.append([sv.rhs_patch(g, e, m) if self.owner[p] == self.rank else np.zeros_like(e)
                       for p, (g, e, m) in enumerate(zip(sv.geos, u[i], mu))])
            new = []
            for p in range(len(sv.geos)):
                acc = np.zeros_like(states[p])
                for k in range(i + 1):
                    if SSP54_ALPHA[i][k] != 0.0:
                        acc = acc + SSP54_ALPHA[i][k] * u[k][p]
                    if SSP54_BETA[i][k] != 0.0:
                        acc = acc + SSP54_BETA[i][k] * dt * Ls[k][p]
                new.append(acc)
            self.project(new)
            u.append(new)
        return u[5], dt


def _rank_main(rank, world, port, owner, wall_form):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import solver as S
        from paper_2506_16076_gb300 import shard, workloads as W
        import dataclasses
        w = W.small_multipatch(W.ADIABATIC)
        w = dataclasses.replace(w, params=dataclasses.replace(w.params, wall_form=wall_form))
        st0 = W.random_smooth_state(w, seed=23, amp=0.05)
        so = ShardedOracle(w, owner, rank, shard.DistComm())
        st, dts = st0, []
        for n in range(NSTEPS):
            st, dt = so.step(st, n)
            dts.append(dt)
        ref, ref_dts = S.Solver(w).run(st0, NSTEPS)
        assert dts == ref_dts, (dts, ref_dts)
        for p, o in enumerate(owner):
            if o == rank:
                assert np.array_equal(st[p], ref[p]), (rank, p, np.abs(st[p] - ref[p]).max())
        assert sum(len(x) for x in so.frecv) > 0 and sum(len(x) for x in so.vrecv) > 0
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("wall_form", [0, 1])
def test_sharded_oracle_steps_over_gloo_equal_single_domain(wall_form):
    # wall_form 1: the product-rule form of the adiabatic wall patch (Remark adiabatic)
    from paper_2506_16076_gb300 import shard, workloads as W
    owner = shard.partition(W.small_multipatch(W.ADIABATIC), 2)
    assert sorted(set(owner)) == [0, 1]
    mp.spawn(_rank_main, args=(2, _free_port(), owner, wall_form), nprocs=2, join=True)
