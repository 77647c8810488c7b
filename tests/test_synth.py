"""The seeded input generators (no method arithmetic): subset sequences are
per-epoch permutations, the detector pitch spans the fan tangent to the
circumscribed circle, phantoms and transmission data are deterministic per seed
and follow their stated recipes, the mixed sweep has its three size classes."""
import math

import numpy as np

from paper_2203_07308_gb300 import synth


def test_subset_sequence_is_one_permutation_per_epoch():
    for P, n in ((8, 100), (12, 30), (5, 5), (3, 7)):
        seq = synth.subset_sequence(n, P, 42)
        assert seq.shape == (n,) and seq.dtype == np.int32
        for e in range(0, n - P + 1, P):
            assert sorted(seq[e:e + P]) == list(range(P))          # every full epoch visits every subset
        assert ((seq >= 0) & (seq < P)).all()
        assert np.array_equal(seq, synth.subset_sequence(n, P, 42))
    assert not np.array_equal(synth.subset_sequence(64, 8, 1), synth.subset_sequence(64, 8, 2))
    assert (synth.subset_sequence(10, 1, 3) == 0).all()
    stages = [synth.Stage(2, 20, 8), synth.Stage(1, 0, 4), synth.Stage(1, 30, 6)]
    seq = synth.schedule_sequence(stages, 9)
    assert seq.shape == (50,) and seq[:20].max() < 8 and seq[20:].max() < 6


def test_flat_detector_pitch_spans_the_tangent_fan():
    for n, nd, dso, ddo in ((256, 512, 512.0, 512.0), (64, 96, 128.0, 64.0), (512, 768, 1024.0, 1024.0)):
        p = synth.flat_detector_pitch(n, nd, dso, ddo)
        half = 0.5 * nd * p                                   # outer edge of the outermost bin
        gamma = math.atan(half / (dso + ddo))
        assert abs(dso * math.sin(gamma) - n / math.sqrt(2.0)) < 1e-9 * n   # edge ray tangent to the circle


def test_ellipse_phantom_recipe():
    a = synth.ellipse_phantom(64, 7)
    assert a.shape == (64, 64) and a.dtype == np.float64
    assert a.min() >= 0.0 and a.max() <= 1.0 and a.max() > 0.0
    assert np.array_equal(a, synth.ellipse_phantom(64, 7))
    assert not np.array_equal(a, synth.ellipse_phantom(64, 8))
    # ellipse centres lie in the disk of radius 0.35 n and semi-axes are at most
    # 0.25 n, so nothing reaches beyond 0.6 n from the centre
    c = np.arange(64) - 31.5
    r = np.hypot(*np.meshgrid(c, c))
    assert (a[r > 0.6 * 64] == 0.0).all()


def test_poisson_transmission_recipe():
    li = np.linspace(0.0, 100.0, 5000)
    b, w = synth.poisson_transmission(li, 10 ** 5.5, 3)
    b2, w2 = synth.poisson_transmission(li, 10 ** 5.5, 3)
    assert np.array_equal(b, b2) and np.array_equal(w, w2)
    mu = 0.02
    counts = w / mu ** 2
    assert np.allclose(counts, np.round(counts)) and counts.min() >= 1.0
    assert np.allclose(b, -np.log(counts / 10 ** 5.5) / mu)
    # high dose: the log data scatter around the line integrals with the Poisson
    # standard deviation 1 / (mu sqrt(counts))
    z = (b - li) * mu * np.sqrt(counts)
    assert abs(z.mean()) < 0.1 and abs(z.std() - 1.0) < 0.1


def test_mixed_classes_cover_the_instances():
    classes = synth.mixed_classes(64)
    sizes = [(wl.geom.n, wl.geom.n_views, wl.geom.n_det) for wl, _ in classes]
    assert sizes == [(128, 180, 256), (256, 360, 512), (512, 720, 768)]
    ids = np.sort(np.concatenate([i for _, i in classes]))
    assert np.array_equal(ids, np.arange(64))
    assert all(wl.geom.batch == len(i) for wl, i in classes)
