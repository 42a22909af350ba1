"""Child process of the bounds-checked build's GPU test: loads
libhcgs_checked.so (HCGS_CHECKED=1) and reports, as one JSON line, what its
checks said in each case."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch
    import hcgs_synth as S
    import oracle
    from gpu_common import cams, cams_dev, complex_dev, dev, oracle_opts, rel
    import paper_2506_08350_b300 as P
    out = {"checked": P.CHECKED, "is_checked_build": int(P._lib.hcgs_is_checked_build())}
    ctx = P.Context(0)

    def status():
        try:
            ctx.check_status()
            return "HCGS_OK"
        except P.HcgsError as e:
            return str(e).split(" ")[0]

    o = S.Optics(48, 80, S.WAVELENGTHS_RGB, (0.0, 2e-3, 4e-3))
    g = S.make_gaussians(800, o.L, o.C, o.H, o.W, seed=4, log_scale_mean=-3.2)
    vm, it = cams(2, o.H, o.W, seed=1)
    vmd, itd = cams_dev(vm, it)
    gd = dev(g)
    holo = torch.empty((2, o.C, o.H, o.W), dtype=torch.complex64, device="cuda")
    saved = P.Saved(ctx)
    ctx.render_view(gd, vmd, itd, o, P.DEFAULT_OPTS, holo, None, saved)
    gP = S.random_complex((2, o.C, o.H, o.W), seed=7)
    grads = {k: torch.empty_like(gd[k]) for k in P.PARAM_NAMES}
    ctx.render_view_backward(saved, gd, complex_dev(gP), grads)
    out["clean_run"] = status()
    oo = oracle_opts(dict(P.DEFAULT_OPTS))
    Po, _, _, _ = oracle.render(g, vm.astype(np.float64), it.astype(np.float64), o, oo)
    out["hologram_rel"] = rel(holo.cpu().numpy(), Po)
    ref = oracle.render_backward(g, vm.astype(np.float64), it.astype(np.float64), o, gP.astype(np.complex128), oo)
    out["grad_rel_max"] = max(rel(grads[k].cpu().numpy(), ref[k]) for k in P.PARAM_NAMES)
    # a failed index check (the index stays inside its buffer)
    ctx.selftest_device_check(0)
    out["index_check"] = status()
    out["after_index_check"] = status()
    # a damaged guard band (inside the allocation); the band is filled again
    ctx.selftest_device_check(1)
    out["guard_band"] = status()
    out["after_guard_band"] = status()
    # a non-finite Gaussian parameter: reported by the projection, at the
    # render's own readback of the status word (after the projection) or at
    # the next hcgs_check_status
    def render_status(gg):
        try:
            ctx.render_view(gg, vmd, itd, o, P.DEFAULT_OPTS, holo, None, saved)
        except P.HcgsError as e:
            return str(e).split(" ")[0]
        return status()

    gn = {k: v.clone() for k, v in gd.items()}
    gn["means"][5, 0] = float("nan")
    out["nan_mean"] = render_status(gn)
    gn = {k: v.clone() for k, v in gd.items()}
    gn["phase"][9, 1] = float("inf")
    out["inf_phase"] = render_status(gn)
    out["clean_again"] = render_status(gd)
    saved.release()
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
