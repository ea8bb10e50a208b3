"""Host-side validation of fc_init_patches: bad descriptors and geometries are rejected
with a status before any device work (no GPU needed)."""
import dataclasses

import pytest

from paper_2506_16076_gb300 import fcsdnn, workloads as W


def _status(w):
    with pytest.raises(fcsdnn.FcError) as ei:
        fcsdnn.Context(w)
    return ei.value.status


def _box(n1, n2, side=(W.DIRICHLET,) * 4, geom=(0.0, 1.0, 0.0, 1.0)):
    fs = (1.4, 1.0, 0.0, 1.0)
    return W.PatchDesc(W.AFFINE, n1, n2, geom, side, bc=(fs,) * 4)


def _wl(patches, **prm):
    return W.Workload("edge", patches, W.Params(**prm), (1.4, 1.0, 0.0, 1.0), "freestream", 1)


def test_too_few_points_is_invalid():
    assert _status(_wl([_box(1, 16)])) == fcsdnn.FC_ERR_INVALID


def test_unknown_patch_kind_is_invalid():
    p = dataclasses.replace(_box(16, 16), kind=7)
    assert _status(_wl([p])) == fcsdnn.FC_ERR_INVALID


def test_wall_on_a_periodic_side_is_invalid():
    w = W.small_multipatch()
    og = w.patches[0]
    bad = dataclasses.replace(og, side=(W.ADIABATIC, og.side[1], og.side[2], og.side[3]))
    assert _status(dataclasses.replace(w, patches=[bad] + w.patches[1:])) == fcsdnn.FC_ERR_INVALID


def test_receivers_without_donor_are_rejected():
    # two boxes with facing internal sides that do not overlap: their fringe points
    # have no donor (donor-receiver condition, Sec. 3.4.1)
    a = _box(32, 32, (W.DIRICHLET, W.INTERNAL, W.DIRICHLET, W.DIRICHLET), (0.0, 1.0, 0.0, 1.0))
    b = _box(32, 32, (W.INTERNAL, W.DIRICHLET, W.DIRICHLET, W.DIRICHLET), (2.0, 3.0, 0.0, 1.0))
    assert _status(_wl([a, b])) == fcsdnn.FC_ERR_DONOR


def test_bad_parameters_are_invalid():
    assert _status(_wl([_box(16, 16)], win_r=0)) == fcsdnn.FC_ERR_INVALID


def _grid_box(side=(W.DIRICHLET,) * 4, **kw):
    return dataclasses.replace(W.as_grid(_box(16, 16, side)), **kw)


def test_grid_patch_with_a_slip_wall_is_invalid():
    assert _status(_wl([_grid_box((W.SLIPWALL,) + (W.DIRICHLET,) * 3)])) == fcsdnn.FC_ERR_INVALID


def test_grid_patch_periodic_on_one_side_only_is_invalid():
    assert _status(_wl([_grid_box((W.PERIODIC,) + (W.DIRICHLET,) * 3)])) == fcsdnn.FC_ERR_INVALID


def test_grid_patch_periodic_in_q2_is_invalid():
    side = (W.DIRICHLET, W.DIRICHLET, W.PERIODIC, W.PERIODIC)
    assert _status(_wl([_grid_box(side)])) == fcsdnn.FC_ERR_INVALID


def test_grid_arrays_of_the_wrong_size_are_rejected_by_the_binding():
    p = _grid_box()
    with pytest.raises(ValueError):
        fcsdnn.Context(_wl([dataclasses.replace(p, metrics=p.metrics[:2])]))


def test_grid_patch_without_metrics_needs_2d_points_per_line():
    # metrics from the points need FC along every non-periodic line
    p = dataclasses.replace(W.as_grid(_box(16, 16)), n1=8, n2=16, metrics=None)
    p = dataclasses.replace(p, x=p.x[:, :8].copy(), y=p.y[:, :8].copy())
    assert _status(_wl([p])) == fcsdnn.FC_ERR_INVALID


def test_free_stream_side_without_a_free_stream_is_invalid():
    # a Dirichlet side of bc density 0 holds fc_params.freestream, which must then be set
    p = dataclasses.replace(_box(16, 16), bc=((0.0, 0.0, 0.0, 0.0),) * 4)
    w = W.Workload("edge", [p], W.Params(), (0.0, 0.0, 0.0, 0.0), "freestream", 1)
    assert _status(w) == fcsdnn.FC_ERR_INVALID


def test_bad_free_stream_is_invalid():
    w = W.Workload("edge", [_box(16, 16)], W.Params(), (1.4, 1.0, 0.0, -1.0), "freestream", 1)
    assert _status(w) == fcsdnn.FC_ERR_INVALID
