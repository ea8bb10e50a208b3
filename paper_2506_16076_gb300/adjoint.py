"""Checkpointed discrete adjoint of the time stepper and a torch.autograd.Function.

The differentiated map is a sequence of fc_rk_step calls with the viscosity and
the time step of each step frozen at their forward values (the smoothness
classifier is not differentiable); with filter=True the per-step filter runs on
steps n >= 1 as in a plain run (Sec. 4.3.1) and is differentiated too. The forward
run stores the state every K steps; the backward run recomputes each segment of K
states from its checkpoint (fc_rk_step with FROZEN_MU | FIXED_DT and the recorded
filter flag, replaying the recorded mu and dt) and applies fc_adjoint_step
backwards through the segment.

Orchestration only: every step and adjoint step runs in the CUDA library.
"""
import torch

from . import fcsdnn


class Trajectory:
    def __init__(self, K):
        self.K = K
        self.checkpoints = {}
        self.mus = []
        self.dts = []
        self.flags = []  # STEP_FILTER or 0, per step


def forward(ctx, e0, nsteps, K, flags=0, filter=False, store_mu=True, first_filtered=1):
    """Run nsteps steps from e0 (not modified); returns (e_N, Trajectory). filter: apply
    the per-step filter on steps n >= first_filtered. store_mu False keeps only the
    checkpoints and the time steps: the backward run then recomputes each step's
    viscosity from the replayed state (the classifier and the viscosity are
    deterministic, so it is the same mu), trading one viscosity evaluation per step for
    P doubles of memory per step."""
    e = e0.clone()
    tr = Trajectory(K)
    tr.checkpoints[0] = e0.clone()
    mu = None
    for n in range(nsteps):
        if store_mu or mu is None:
            mu = torch.empty(ctx.P, dtype=torch.float64, device=e.device)
        dt = torch.zeros(1, dtype=torch.float64, device=e.device)
        f = fcsdnn.STEP_FILTER if (filter and n >= first_filtered) else 0
        ctx.rk_step(e, dt, mu, (flags & ~fcsdnn.STEP_FILTER) | f)
        tr.mus.append(mu if store_mu else None)
        tr.dts.append(dt)
        tr.flags.append(f)
        if (n + 1) % K == 0 and n + 1 < nsteps:
            tr.checkpoints[n + 1] = e.clone()
    return e, tr


def replay(ctx, tr, e0, n0, n1):
    """States e_{n0}..e_{n1-1} recomputed from e_{n0} with the recorded dt and filter flag
    and the recorded (or recomputed) mu; returns (states, mus)."""
    out = [e0.clone()]
    mus = []
    e = e0.clone()
    for n in range(n0, n1):
        mu = tr.mus[n]
        if mu is None:  # the forward viscosity of step n: from its projected input state
            mu = torch.empty(ctx.P, dtype=torch.float64, device=e.device)
            ep = e.clone()
            ctx.project(ep)
            ctx.viscosity(ep, mu)
            del ep
        mus.append(mu)
        if n < n1 - 1:
            ctx.rk_step(e, tr.dts[n], mu, fcsdnn.STEP_FROZEN_MU | fcsdnn.STEP_FIXED_DT | tr.flags[n])
            out.append(e.clone())
    return out, mus


def backward(ctx, tr, lam_N, dparam=None):
    """lam_0 = (d e_N / d e_0)^T lam_N and the accumulated Dirichlet sensitivity gbc; dparam
    (2 device doubles, optional) accumulates dJ/d(Mach, angle) through the free-stream
    Dirichlet states of every step."""
    nsteps = len(tr.dts)
    lam = lam_N.clone()
    nxt = torch.empty_like(lam)
    gbc = torch.zeros_like(lam)
    starts = sorted(tr.checkpoints)
    for si in range(len(starts) - 1, -1, -1):
        n0 = starts[si]
        n1 = starts[si + 1] if si + 1 < len(starts) else nsteps
        states, mus = replay(ctx, tr, tr.checkpoints[n0], n0, n1)
        for n in range(n1 - 1, n0 - 1, -1):
            ctx.adjoint_step(states[n - n0], mus[n - n0], tr.dts[n], lam, nxt, gbc, tr.flags[n], dparam)
            lam, nxt = nxt, lam
        del states, mus
    return lam, gbc


class FCSteps(torch.autograd.Function):
    """e_N = steps(e_0): forward through fc_rk_step, backward through fc_adjoint_step."""

    @staticmethod
    def forward(fctx, e0, ctx, nsteps, K):
        eN, tr = forward(ctx, e0, nsteps, K)
        fctx.ctx, fctx.tr = ctx, tr
        return eN

    @staticmethod
    def backward(fctx, grad):
        lam0, gbc = backward(fctx.ctx, fctx.tr, grad.contiguous())
        fctx.gbc = gbc
        return lam0, None, None, None


def drag(ctx, e):
    J = torch.zeros(1, dtype=torch.float64, device=e.device)
    g = torch.zeros_like(e)
    ctx.drag(e, J, g)
    return J, g


def drag_gradients(w, ctx, e0, nsteps, K, filter=False):
    """J after nsteps from the free-stream state e0 and dJ/dMach, dJ/dangle, dJ/drho_0(x).

    Mach and angle enter through the initial state and the Dirichlet free-stream
    states (fc_adjoint_step and fc_initial_sensitivity accumulate both parts on the
    device); rho_0 perturbs the initial density at fixed velocity and pressure."""
    eN, tr = forward(ctx, e0, nsteps, K, filter=filter)
    J, dJde = drag(ctx, eN)
    dparam = torch.zeros(2, dtype=torch.float64, device=e0.device)
    lam0, _ = backward(ctx, tr, dJde, dparam)
    dJdrho = torch.empty(e0.shape[1], dtype=torch.float64, device=e0.device)
    ctx.initial_sensitivity(e0, lam0, dJdrho, dparam)
    dJdM, dJda = dparam.tolist()
    return J.item(), dJdM, dJda, dJdrho, tr
