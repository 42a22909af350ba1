"""Helpers shared by the GPU parity tests (inputs come from hcgs_synth only)."""
import numpy as np

import hcgs_synth as S

PARAMS = ("means", "log_scales", "quats", "opacity_logits", "amplitude", "phase", "plane_logits")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(g):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(g[k], dtype=np.float32)).cuda() for k in PARAMS}


def cams(V, H, W, seed=0):
    """float32 cameras (the oracle gets the same float32-rounded values)."""
    vm, it = S.view_batch(V, H, W, seed=seed)
    return vm.astype(np.float32), it.astype(np.float32)


def cams_dev(vm, it):
    import torch
    return torch.from_numpy(vm).cuda().contiguous(), torch.from_numpy(it).cuda().contiguous()


def complex_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


ORACLE_OPTS_OF = {"alpha_min": "alpha_min", "alpha_max": "alpha_max", "T_eps": "T_eps",
                  "cov2d_dilation": "dilation", "near_z": "near_z", "clip_factor": "clip", "order": "order",
                  "ste_tau": "tau"}


def oracle_opts(gpu_opts):
    """The oracle's option dict for a GPU option dict (same thresholds, as
    float32-rounded values)."""
    out = {}
    for k, v in gpu_opts.items():
        if k in ORACLE_OPTS_OF:
            out[ORACLE_OPTS_OF[k]] = float(np.float32(v)) if k != "order" else int(v)
    return out
