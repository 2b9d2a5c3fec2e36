"""The seeded synthetic workload: shapes, determinism and the structure the
recipe promises (corridor path, spacing, aliasing, windows)."""
import numpy as np

import synth


def test_path_spacing_and_nonnegative_coordinates():
    arc = 0.5 * np.arange(2000)
    xy = synth.path_positions(arc)
    steps = np.hypot(*np.diff(xy, axis=0).T)
    # 0.5 m everywhere except where a step turns a corridor corner (shorter chord)
    assert np.all(steps <= 0.5 + 1e-9) and np.mean(np.isclose(steps, 0.5)) > 0.97
    assert xy.min() >= 1.0 - 1e-12
    # parallel corridors 3 m apart: away from the corridor ends, y takes only
    # the values 1 + 3c
    inner = (xy[:, 0] > 1.0 + 1e-9) & (xy[:, 0] < 101.0 - 1e-9)
    ys = np.unique(np.round(xy[inner, 1], 9))
    assert np.allclose(np.diff(ys), 3.0) and ys.size == 10


def test_database_is_deterministic_and_shaped():
    a = synth.make_database(3000, 128, seed=1000)
    b = synth.make_database(3000, 128, seed=1000)
    assert a.feats.dtype == np.float32 and a.feats.shape == (3000, 128)
    assert a.xy.dtype == np.float64 and a.xy.shape == (3000, 2)
    assert np.array_equal(a.feats, b.feats) and np.array_equal(a.xy, b.xy)
    c = synth.make_database(3000, 128, seed=1001)
    assert not np.array_equal(a.feats, c.feats)
    # unit-variance field
    assert 0.8 < float(a.feats.std()) < 1.2


def test_scene_aliasing_fraction_and_distance():
    db = synth.make_database(5000, 64, seed=3)
    assert abs(db.aliased.mean() - 0.10) < 0.005
    rows = np.nonzero(db.aliased)[0]
    src = db.alias_src[rows]
    assert np.all(np.hypot(*(db.xy[src] - db.xy[rows]).T) >= 10.0)
    base = db.field(db.xy[src])
    resid = db.feats[rows] - base
    assert 0.008 < float(resid.std()) < 0.012


def test_field_is_smooth_over_the_correlation_length():
    db = synth.make_database(2000, 128, seed=4, alias_frac=0.0)
    # neighbours 0.5 m apart are strongly correlated, points 20 m apart are not
    f = db.feats.astype(np.float64)
    near = np.mean(np.sum(f[1:] * f[:-1], 1) / np.sum(f[1:] ** 2, 1))
    far = np.mean(np.sum(f[40:] * f[:-40], 1) / np.sum(f[40:] ** 2, 1))
    assert near > 0.9 and abs(far) < 0.3


def test_point_queries():
    db = synth.make_database(2000, 128, seed=1000)
    q, rows, txy = synth.make_point_queries(db, 16, seed=2000)
    assert q.shape == (16, 128) and q.dtype == np.float32
    assert np.array_equal(txy, db.xy[rows])
    noise = q - db.feats[rows]
    assert 0.04 < float(noise.std()) < 0.06


def test_windows_layout():
    db = synth.make_database(4000, 64, seed=5)
    w = synth.make_windows(db, 7, 5, seed=6)
    assert w.offsets.tolist() == [0, 5, 10, 15, 20, 25, 30, 35]
    assert w.frames.shape == (35, 64) and w.frames.dtype == np.float32
    # frames 0.3 m apart along the path, the reference is frame floor(m/2)
    for i in range(7):
        fx = w.frame_xy[w.offsets[i]:w.offsets[i + 1]]
        assert np.all(np.hypot(*np.diff(fx, axis=0).T) <= 0.3 + 1e-9)
        assert np.array_equal(w.true_xy[i], fx[2])
    u = synth.make_windows(db, 50, (3, 10), seed=7)
    lens = u.lengths()
    assert lens.min() >= 3 and lens.max() <= 10 and len(set(lens.tolist())) > 3
