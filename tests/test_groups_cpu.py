"""Host logic of the shot groups (no GPU): a group's acquisition keeps exactly
its shots' sources, wavelets, moment tensors or forces, windows and traces, in
order, and the groups together cover every trace once."""
import numpy as np

import workloads as W


def test_group_acquisition_slices_every_per_shot_array():
    from paper_2305_14130_gb300.groups import group_acquisition
    p = W.with_forces(W.tiny(nx=48, nz=26, ns=5, nt=20, npml=4,
                             win=[[0, 30], [9, 37], [20, 28], [4, 40], [12, 30]]))
    a = p.acq
    seen = []
    for shots in ([0, 1], [2, 3], [4]):
        g, idx = group_acquisition(a, shots)
        assert np.array_equal(g.src_xz, a.src_xz[shots]) and np.array_equal(g.mt, a.mt[shots])
        assert np.array_equal(g.wavelet, a.wavelet[shots]) and np.array_equal(g.force, a.force[shots])
        assert np.array_equal(g.win, np.asarray(a.win)[shots])
        counts = [int(a.tr_ptr[s + 1] - a.tr_ptr[s]) for s in shots]
        assert list(np.diff(g.tr_ptr)) == counts and g.tr_ptr[0] == 0
        expect = np.concatenate([np.arange(a.tr_ptr[s], a.tr_ptr[s + 1]) for s in shots])
        assert np.array_equal(idx, expect)
        assert np.array_equal(g.ch_xz, a.ch_xz[idx]) and np.array_equal(g.ch_t, a.ch_t[idx])
        assert (g.nx, g.nz, g.nt, g.dt, g.gauge) == (a.nx, a.nz, a.nt, a.dt, a.gauge)
        seen.append(idx)
    assert np.array_equal(np.concatenate(seen), np.arange(a.ntr))
