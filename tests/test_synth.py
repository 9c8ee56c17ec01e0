"""The synthetic-input fixture: shape, determinism and the sharing it promises."""
import numpy as np

import synth


def test_descriptor_recipe_statistics():
    w = synth.pair2k()
    d, kp, tr = w.generate(want_kp=True, want_track=True)
    assert d.shape == (4000, 128) and d.dtype == np.uint8
    norms = np.linalg.norm(d.astype(np.float64), axis=1)
    # |N(0,1)| normalised and scaled to 255: norm ~255, per-dimension mean ~18
    assert abs(np.median(norms[:2000]) - 255) < 3
    assert 16 < d.mean() < 20
    # 40 % of B observes tracks that A holds exactly (A's sigma is 0)
    a, b = tr[:2000], tr[2000:]
    assert (a >= 0).sum() == 800 and (b >= 0).sum() == 800
    assert set(a[a >= 0]) == set(b[b >= 0])
    pos_a = {t: k for k, t in enumerate(a) if t >= 0}
    diff = np.array([d[2000 + k].astype(int) - d[pos_a[t]].astype(int) for k, t in enumerate(b) if t >= 0])
    # sigma-8 noise, a little less after clipping at 0
    assert 6.5 < diff.std() < 8.5 and abs(diff.mean()) < 1.5


def test_generation_is_deterministic_and_sliceable():
    w = synth.strip30(n_images=6, n=500)
    full = w.generate(threads=3)
    part = w.generate(2, 4, threads=1)
    off = w.row_off
    assert np.array_equal(full[off[2]:off[4]], part)
    assert np.array_equal(full, w.generate(threads=1))


def test_workload_shapes():
    assert len(synth.strip30().pairs) == 120
    g = synth.grid500()
    assert g.n_images == 500 and 2000 <= g.n_desc.min() and g.n_desc.max() <= 20000
    assert len(g.pairs) == 2777 and np.all(g.pairs[:, 0] < g.pairs[:, 1])
    o = synth.oblique200()
    assert o.n_images == 200 and len(o.pairs) == 3200
    big = synth.grid5000()
    assert big.n_images == 5000 and len(big.pairs) == 58504 and big.total_desc == 100_000_000
    for wl in (synth.strip30(), g, o, big):
        fr = wl.shared_fraction()
        assert 0.2 <= fr.mean() <= 0.4
