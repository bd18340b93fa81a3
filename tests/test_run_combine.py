"""The run form of the warp-combined adjoint, simulated lane by lane on the
CPU.

Per plane, lane k of a warp holds a z voxel index ib_k and two taps: g0 to
voxel ib_k and g1 to voxel ib_k + 1.  When no three neighbouring lanes
share a voxel, the kernel combines the taps by runs (one or two lanes on
one voxel, walked in z order) so that every voxel gets exactly one write.
This test restates those rules with the kernel's shuffle semantics (a
source lane is taken modulo 32) and checks, on random run patterns with
gaps, in both z orders, that the writes sum to direct tap-by-tap
accumulation and that no voxel is written twice.
"""
import numpy as np
import pytest


def run_form(ib, g0, g1, asc):
    """Writes (voxel, value) made by the 32 lanes under the run form."""
    lanes = np.arange(32)
    prev = (lanes - 1 if asc else lanes + 1) & 31
    nxt = (lanes + 1 if asc else lanes - 1) & 31
    has_prev = lanes > 0 if asc else lanes < 31
    has_next = lanes < 31 if asc else lanes > 0
    dn = np.where(has_next, ib[nxt] - ib, 2)
    up = np.where(has_prev, ib - ib[prev], 2)
    e1 = np.where(up == 0, g1 + g1[prev], g1)
    s0 = np.where(dn == 0, g0 + g0[nxt], g0)
    x0 = np.where(up == 1, s0 + e1[prev], s0)
    w0 = up != 0
    w1 = (dn.astype(np.int64) & 0xFFFFFFFF) > 1          # unsigned compare, as in the kernel
    writes = [(int(ib[k]), float(x0[k])) for k in lanes if w0[k]]
    writes += [(int(ib[k]) + 1, float(e1[k])) for k in lanes if w1[k]]
    return writes


def random_pattern(rng, asc):
    """ib for 32 lanes in z order: steps of 0 (two lanes on a voxel, never
    twice in a row), 1, or a gap of 2..4 voxels."""
    steps = []
    for _ in range(31):
        s = rng.choice([0, 1, 1, 1, 2, 3, 4], p=[0.25, 0.15, 0.15, 0.15, 0.15, 0.1, 0.05])
        if s == 0 and steps and steps[-1] == 0:
            s = 1
        steps.append(int(s))
    z = 1000 + np.concatenate([[0], np.cumsum(steps)])
    return z if asc else z[::-1].copy()


@pytest.mark.parametrize("asc", [True, False])
def test_run_form_equals_direct_accumulation(asc):
    rng = np.random.default_rng(31 + asc)
    for _ in range(2000):
        ib = random_pattern(rng, asc)
        # lanes two apart differ by at least one voxel (the kernel's run check)
        d = ib[2:] - ib[:-2]
        assert (d >= 1).all() if asc else (d <= -1).all()
        g0 = rng.standard_normal(32)
        g1 = rng.standard_normal(32)
        direct = {}
        for k in range(32):
            direct[ib[k]] = direct.get(ib[k], 0.0) + g0[k]
            direct[ib[k] + 1] = direct.get(ib[k] + 1, 0.0) + g1[k]
        writes = run_form(ib, g0, g1, asc)
        voxels = [v for v, _ in writes]
        assert len(voxels) == len(set(voxels)), "a voxel written twice"
        got = dict(writes)
        assert set(got) == set(direct)
        for v in direct:
            assert abs(got[v] - direct[v]) <= 1e-12 * (1 + abs(direct[v]))


def test_run_form_halves_writes_for_unit_spacing():
    """Rays one voxel apart: 33 writes per row for 32 lanes in either z
    order (each voxel once), against 64 for tap-by-tap scatter."""
    for asc in (True, False):
        ib = 500 + np.arange(32)
        if not asc:
            ib = ib[::-1].copy()
        writes = run_form(ib, np.ones(32), np.ones(32), asc)
        assert len(writes) == 33
