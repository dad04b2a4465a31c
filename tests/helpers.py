"""Shared test helpers: move seeded workloads to the GPU and compare with the oracle.

Relative errors follow Eq. L2_norm_error (Sec. 5.2): ||a - b|| / ||b||, with the
norm of a field taken over its three components together (a component that is
identically zero in the reference is compared against the size of its field).
"""
import numpy as np

TOL = 1e-12          # FP64 parity tolerance (relative L2)


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def field_rel_err(gpu, ref):
    """max over components of ||g_c - r_c|| / max_c ||r_c||."""
    scale = max(float(np.linalg.norm(r)) for r in ref)
    if scale == 0.0:
        scale = 1.0
    return max(float(np.linalg.norm(np.asarray(g) - np.asarray(r))) / scale for g, r in zip(gpu, ref))


def species_to_dev(sp_list, with_id=True):
    import torch
    from paper_2106_12919_gb300 import pic
    out = []
    for s in sp_list:
        n = s["x"].size
        ident = torch.arange(n, dtype=torch.int64, device="cuda") if with_id else None
        out.append(pic.Species(to_dev(s["x"]), to_dev(s["y"]), to_dev(s["z"]), to_dev(s["ux"]), to_dev(s["uy"]),
                               to_dev(s["uz"]), to_dev(s["w"]), s["q"], s["m"], id=ident))
    return out


def species_from_dev(sp_dev):
    """Back to host dicts in the original particle order (using the id tag)."""
    out = []
    for s in sp_dev:
        order = np.argsort(to_host(s.id))
        d = {k: to_host(getattr(s, k))[order] for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
        d["q"], d["m"] = s.q, s.m
        out.append(d)
    return out


def context_for(params, **kw):
    from paper_2106_12919_gb300 import pic
    p = dict(params)
    return pic.Context(p["shape"], p["dx"], p["dt"], p["shape_order"], p["centering_order"], p["variant"],
                       p["v_gal"], p["spectral_order"], p["c"], p["eps0"], **kw)


def periodic_pos_err(a, b, L):
    d = np.abs(a - b)
    return np.minimum(d, L - d)
