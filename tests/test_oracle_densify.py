"""Pins for the oracle's densification (Algorithm 1: pruning, phase-aware
clone and split) and for the counter-based generator that draws its noise.

The generator is pinned to the known-answer vectors published with the
reference implementation of Philox4x32-10 (Salmon et al., SC'11, Random123),
its normals to the standard normal distribution; the densification rules to
hand-built cases whose decisions follow from the thresholds, and the split
children to the distribution they are drawn from (covariance R diag(s^2) R^T
with R from scipy's quaternion routine)."""
import math

import numpy as np
from scipy import stats
from scipy.spatial.transform import Rotation

import oracle


def test_philox_known_answers():
    kat = [(([0, 0, 0, 0], [0, 0]), [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
           (([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2), [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
           (([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]),
            [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1])]
    for (ctr, key), want in kat:
        assert list(oracle.philox4x32_10(ctr, key)) == want


def test_philox_streams_are_distinct_and_uniform():
    a = oracle.philox_words(7, 200_000, stream=0)
    b = oracle.philox_words(7, 200_000, stream=1)
    c = oracle.philox_words(8, 200_000, stream=0)
    assert np.mean(a == b) < 1e-3 and np.mean(a == c) < 1e-3
    # the top byte is uniform over 256 values
    counts = np.bincount(a >> 24, minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4


def test_uniform_map_is_the_open_interval_symmetric_about_one_half():
    # the word -> uniform map: centres of the 2^32 cells of [0, 1).  The ends
    # stay inside (0, 1), and u(w) + u(2^32 - 1 - w) = 1 exactly, which the
    # map w 2^-32 (or (w + 1) 2^-32) breaks by 2^-32
    top = 2 ** 32 - 1
    w = np.array([0, 1, 2 ** 23 - 1, 2 ** 31 - 1, 2 ** 31, top - 5, top], dtype=np.uint32)
    u = oracle.uniform_of_words(w)
    assert u[0] == 2.0 ** -33 and u[-1] == 1.0 - 2.0 ** -33
    assert np.all((u > 0) & (u < 1)) and np.all(np.diff(u) > 0)
    assert np.array_equal(u + oracle.uniform_of_words(top - w.astype(np.int64)), np.ones(w.size))
    # and it is what the uniforms of a stream are made of
    assert np.array_equal(oracle.philox_uniforms(3, 9, 2), oracle.uniform_of_words(oracle.philox_words(3, 9, 2)))


def test_philox_normals_are_standard_normal():
    z = oracle.philox_normals(11, 400_000)
    assert abs(z.mean()) < 5 * 1.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # odd counts end inside a pair
    assert np.array_equal(oracle.philox_normals(11, 5), z[:5])


def _gauss(n, C=3, L=4):
    return dict(means=np.zeros((n, 3)), log_scales=np.full((n, 3), math.log(0.01)), quats=np.tile([1.0, 0, 0, 0], (n, 1)),
                opacity_logits=np.zeros(n), amplitude=np.ones((n, C)), phase=np.zeros((n, C)),
                plane_logits=np.zeros((n, L)))


def test_actions_follow_the_thresholds():
    g = _gauss(7)
    o = dict(oracle.DENSIFY_OPTS, prune_scale=0.5)
    g["opacity_logits"][1] = math.log(0.004 / 0.996)          # opacity 0.004 < 0.005: pruned
    g["log_scales"][3, 2] = math.log(0.05)                    # largest scale 0.05 > split_scale 0.02
    g["log_scales"][4, 0] = math.log(0.8)                     # larger than prune_scale: pruned
    accum = np.array([1e-4, 1.0, 3e-4, 3e-4, 3e-4, 0.0, 2.1e-4], dtype=np.float32)
    denom = np.array([1, 1, 1, 1, 1, 0, 1], dtype=np.float32)
    act = oracle.densify_actions(g, accum, denom, o)
    assert list(act) == [oracle.KEEP, oracle.PRUNE, oracle.CLONE, oracle.SPLIT, oracle.PRUNE, oracle.KEEP,
                         oracle.CLONE]
    # the mean over views decides: 3e-4 over two views is below the threshold
    denom2 = denom.copy()
    denom2[2] = 2
    assert oracle.densify_actions(g, accum, denom2, o)[2] == oracle.KEEP


def test_densify_counts_order_and_copies():
    rng = np.random.default_rng(0)
    n, C = 200, 3
    g = _gauss(n, C)
    g["means"] = rng.normal(size=(n, 3))
    g["log_scales"] = rng.normal(-4.0, 0.6, size=(n, 3))
    g["quats"] = rng.normal(size=(n, 4))
    g["opacity_logits"] = rng.normal(0.0, 3.0, size=n)
    g["phase"] = rng.uniform(0, 2 * np.pi, size=(n, C))
    g["plane_logits"] = rng.normal(size=(n, 4))
    accum = rng.uniform(0, 6e-4, size=n).astype(np.float32)
    denom = rng.integers(0, 3, size=n).astype(np.float32)
    noise = rng.normal(size=(n, 2, 3 + C))
    m = rng.normal(size=(n, 3))
    newp, (newm,), act = oracle.densify(g, accum, denom, noise, extra=(m,))
    per = np.array([1, 0, 2, 2])[act]
    assert newp["means"].shape[0] == per.sum() == newm.shape[0]
    assert set(act) == {oracle.KEEP, oracle.PRUNE, oracle.CLONE, oracle.SPLIT}
    off = np.concatenate([[0], np.cumsum(per)])
    for i in range(n):
        j = off[i]
        if act[i] in (oracle.KEEP, oracle.CLONE):
            for k in g:
                assert np.array_equal(newp[k][j], g[k][i])
            assert np.array_equal(newm[j], m[i])
        if act[i] == oracle.CLONE:
            for k in g:
                want = g[k][i] + (0.1 * noise[i, 0, 3:] if k == "phase" else 0.0)
                assert np.allclose(newp[k][j + 1], want, rtol=0, atol=1e-15)
            assert np.all(newm[j + 1] == 0)
        if act[i] == oracle.SPLIT:
            for c in range(2):
                assert np.allclose(newp["log_scales"][j + c], g["log_scales"][i] - math.log(1.6))
                assert np.allclose(newp["phase"][j + c], g["phase"][i] + 0.1 * noise[i, c, 3:])
                for k in ("quats", "opacity_logits", "amplitude", "plane_logits"):
                    assert np.array_equal(newp[k][j + c], g[k][i])
                assert np.all(newm[j + c] == 0)


def test_split_children_are_draws_from_the_parent():
    # one anisotropic rotated Gaussian split many times: the children's means
    # have mean mu and covariance R diag(s^2) R^T
    q = np.array([0.8, 0.3, -0.4, 0.2])
    s = np.array([0.05, 0.02, 0.01])
    K = 40_000
    g = _gauss(K)
    g["means"][:] = [0.3, -0.2, 2.0]
    g["log_scales"][:] = np.log(s)
    g["quats"][:] = q
    accum = np.full(K, 1.0, dtype=np.float32)
    denom = np.ones(K, dtype=np.float32)
    noise = np.random.default_rng(1).normal(size=(K, 2, 6))
    newp, _, act = oracle.densify(g, accum, denom, noise)
    assert np.all(act == oracle.SPLIT)
    d = newp["means"] - g["means"][0]
    Rs = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    cov = Rs @ np.diag(s ** 2) @ Rs.T
    emp = d.T @ d / d.shape[0]
    assert np.max(np.abs(d.mean(0))) < 5 * s.max() / math.sqrt(d.shape[0])
    assert np.max(np.abs(emp - cov)) < 6 * s.max() ** 2 * math.sqrt(2.0 / d.shape[0])


def test_accumulate_uses_ndc_gradient_norm_of_visible_gaussians():
    gmu = np.array([[3.0, 4.0], [1.0, 0.0], [0.0, 2.0]])
    valid = np.array([1, 0, 1])
    a, d = oracle.densify_accumulate(np.zeros(3), np.zeros(3), valid, gmu, H=10, W=20)
    assert np.allclose(a, [math.hypot(3 * 10, 4 * 5), 0.0, 10.0])
    assert list(d) == [1.0, 0.0, 1.0]
