"""The seeded synthetic inputs follow the stated recipes (no GPU): the
Gaussian random field has the power-law spectrum it is built with, the
log-normal particles sample exp(g), the batch specification draws counts
log-uniformly with half uniform and half clumpy snapshots, and the same seed
gives the same particles."""
import numpy as np

import synth


def test_grf_spectrum_slope_and_mean():
    rng = np.random.default_rng(3)
    g = synth.gaussian_random_field(64, -4.0, rng)
    assert abs(g.mean()) < 1e-12
    pk = np.abs(np.fft.fftn(g)) ** 2
    k = np.fft.fftfreq(64) * 64
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    bins = np.arange(2, 20)
    p = np.array([pk[(kk >= b) & (kk < b + 1)].mean() for b in bins])
    slope = np.polyfit(np.log(bins + 0.5), np.log(p), 1)[0]
    assert abs(slope + 4.0) < 0.3, slope


def test_lognormal_particles_sample_exp_g():
    """Counts per voxel of the field grid follow rho ~ exp(g): the densest
    tenth of voxels holds far more than a tenth of the particles, and the
    spread of log counts in occupied coarse cells grows with sigma."""
    spread = []
    for sigma in (0.5, 1.5):
        p = synth.lognormal_particles(200000, 11, sigma=sigma, ngrid=32)
        assert np.all((p.pos() >= 0) & (p.pos() < 1)) and abs(p.m.sum() - 1) < 1e-12
        c = np.floor(p.pos() * 8).astype(int)
        counts = np.bincount((c[:, 0] * 8 + c[:, 1]) * 8 + c[:, 2], minlength=512)
        spread.append(np.std(np.log(counts[counts > 0])))
    assert spread[1] > 1.5 * spread[0], spread


def test_batch_specs_and_seeds():
    specs = synth.batch_specs(256, 7)
    n = np.array([s[0] for s in specs])
    kinds = [s[1] for s in specs]
    sig = np.array([s[2] for s in specs])
    assert n.min() >= 2 ** 10 and n.max() <= 2 ** 18
    assert kinds.count("uniform") == kinds.count("clumpy") == 128
    assert np.all((sig >= 1.0) & (sig <= 2.0))
    # log-uniform: the median count near the geometric middle 2^14
    assert 2 ** 13 < np.median(n) < 2 ** 15
    a = synth.lognormal_particles(1000, 5, ngrid=16)
    b = synth.lognormal_particles(1000, 5, ngrid=16)
    assert np.array_equal(a.pos(), b.pos())
