"""The bounds-checked build (libhcgs_checked.so) on the GPU, and the regular
build's handling of out-of-range shapes and non-finite inputs.

The checked build stands in for a memory checker: its kernels check the
indices they take from data before using them, the projection checks that
every parameter is finite, and every library buffer carries a guard band;
hcgs_check_status reports what failed as HCGS_ERR_DEVICE_CHECK and leaves the
context usable.  The failures here are made on purpose without any access
leaving its allocation: an index outside its checked range but inside its
buffer, a byte written into a guard band, NaN and inf inputs.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import hcgs_synth as S
from gpu_common import cams, cams_dev, dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2506_08350_b300 as P
    return P


def test_checked_build_reports_each_failed_check(P):
    env = dict(os.environ, HCGS_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_worker.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    print(out)
    assert out["checked"] and out["is_checked_build"] == 1
    # no check fails on a correct run, and its results are the regular ones
    assert out["clean_run"] == "HCGS_OK"
    assert out["hologram_rel"] < 1e-4 and out["grad_rel_max"] < 1e-3
    for case in ("index_check", "guard_band", "nan_mean", "inf_phase"):
        assert out[case] == "HCGS_ERR_DEVICE_CHECK", (case, out[case])
    # each report clears the word; the context keeps working
    assert out["after_index_check"] == out["after_guard_band"] == out["clean_again"] == "HCGS_OK"


def test_regular_build_culls_a_gaussian_with_a_non_finite_mean(P):
    # without the checks a Gaussian whose mean is not finite fails the
    # near-plane test and is culled: the fields equal those of the scene
    # without it, bit for bit
    o = S.Optics(48, 80, S.WAVELENGTHS_RGB[:2], (0.0, 3e-3))
    g = S.make_gaussians(500, o.L, o.C, o.H, o.W, seed=8, log_scale_mean=-3.2)
    vm, it = cams(1, o.H, o.W, seed=2)
    vmd, itd = cams_dev(vm, it)
    ctx = P.Context(0)
    assert not P.CHECKED and P._lib.hcgs_is_checked_build() == 0

    def planes(gg):
        gd = dev(gg)
        U = torch.empty((1, o.L, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
        h = torch.empty((1, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
        ctx.render_view(gd, vmd, itd, o, P.DEFAULT_OPTS, h, U)
        torch.cuda.synchronize()
        return U.cpu().numpy()

    bad = {k: v.copy() for k, v in g.items()}
    bad["means"][7, 2] = np.nan
    without = {k: np.delete(v, 7, axis=0) for k, v in g.items()}
    Ub, Uw = planes(bad), planes(without)
    ctx.check_status()
    ctx.close()
    assert np.all(np.isfinite(Ub)) and np.array_equal(Ub, Uw)


def test_out_of_range_shapes_are_rejected_before_any_launch(P):
    ctx = P.Context(0)
    g = S.make_gaussians(10, 2, 1, 32, 32, seed=1)
    gd = dev(g)
    vm, it = cams(1, 32, 32)
    vmd, itd = cams_dev(vm, it)
    cases = [(S.Optics(32, 32, (515e-9,) * 5, (0.0, 1e-3)), "INVALID_ARG"),          # C = 5 > 4
             (S.Optics(32, 32, (515e-9,), tuple(np.linspace(0, 1e-2, 17))), "INVALID_ARG"),  # L = 17 > 16
             (S.Optics(32, 7 * 7, (515e-9,), (0.0, 1e-3)), "UNSUPPORTED_SIZE"),       # 49 = 7^2
             (S.Optics(32, 8192, (515e-9,), (0.0, 1e-3)), "UNSUPPORTED_SIZE"),        # longer than 4096
             (S.Optics(32, 32, (-515e-9,), (0.0, 1e-3)), "INVALID_ARG")]              # negative wavelength
    for o, want in cases:
        h = torch.empty((1, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
        with pytest.raises(P.HcgsError, match=want):
            ctx.render_view(gd, vmd, itd, o, P.DEFAULT_OPTS, h)
    # an option out of range
    o = S.Optics(32, 32, (515e-9,), (0.0, 1e-3))
    h = torch.empty((1, 1, 32, 32), dtype=torch.complex64, device="cuda")
    for bad in (dict(footprint=3), dict(order=2), dict(alpha_min=0.5, alpha_max=0.4), dict(tile=8)):
        with pytest.raises(P.HcgsError, match="INVALID_ARG"):
            ctx.render_view(gd, vmd, itd, o, dict(P.DEFAULT_OPTS, **bad), h)
    ctx.check_status()
    ctx.close()
