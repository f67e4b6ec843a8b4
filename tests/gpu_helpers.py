"""Shared helpers for the GPU parity tests (test infrastructure only)."""
import numpy as np
import torch

import oracle
import rs_inputs as ri

_built = False


def rs():
    """The product binding, built for sm_103a if needed (fails loudly without the library)."""
    global _built
    if not _built:
        import __graft_entry__
        __graft_entry__._builder().build()
        _built = True
    import paper_0905_2453_gb300 as m
    return m


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def shoot_gpu(field_spec, grid=None, window=None, rows=None, counts=None, oow=None):
    """GPU counts (numpy uint32 [npix1, npix0]) and out-of-window count of a rs_inputs.Field."""
    m = rs()
    grid = grid or field_spec.grid
    window = window or field_spec.window
    f = m.Field.from_spec(field_spec)
    try:
        if counts is None:
            counts = torch.zeros((int(window.npix[1]), int(window.npix[0])), dtype=torch.int32, device=dev())
        if oow is None:
            oow = torch.zeros(1, dtype=torch.int64, device=dev())
        f.shoot(grid, window, counts, oow, rows=rows)
        torch.cuda.synchronize()
        assert f.status() == m.RS_OK
    finally:
        f.close()
    return counts.cpu().numpy().view(np.uint32), int(oow.item())


def trace_gpu(field_spec, ray_ij, grid=None, chunk=1 << 22, certified=False):
    """float32-path source positions and band half-widths (or float-float positions if certified)."""
    m = rs()
    grid = grid or field_spec.grid
    f = m.Field.from_spec(field_spec)
    try:
        ij = np.asarray(ray_ij, np.int64).reshape(-1, 2)
        ys, es = [], []
        for s in range(0, ij.shape[0], chunk):
            t = torch.from_numpy(ij[s:s + chunk])
            if certified:
                ys.append(f.trace(grid, t, certified=True).cpu().numpy())
            else:
                y, e = f.trace(grid, t, with_err=True)
                ys.append(y.cpu().numpy())
                es.append(e.cpu().numpy())
        torch.cuda.synchronize()
    finally:
        f.close()
    return np.concatenate(ys), (np.concatenate(es) if es else None)


def all_rays(grid, rows=None):
    n0, n1 = int(grid.n[0]), int(grid.n[1])
    jb, je = rows or (0, n1)
    jj, ii = np.meshgrid(np.arange(jb, je, dtype=np.int64), np.arange(n0, dtype=np.int64), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], 1)


def pixel_index(y, window):
    """Pixel index per ray (-1 out of window) with the binning rule of the method (test-side copy)."""
    lo = np.asarray(window.lo, np.float64)
    hi = np.asarray(window.hi, np.float64)
    npix = np.asarray(window.npix, np.float64)
    scale = npix / (hi - lo)
    u = (y - lo[None, :]) * scale[None, :]
    ok = (u[:, 0] >= 0) & (u[:, 0] < npix[0]) & (u[:, 1] >= 0) & (u[:, 1] < npix[1])
    p = np.full(y.shape[0], -1, np.int64)
    p[ok] = np.floor(u[ok, 1]).astype(np.int64) * int(window.npix[0]) + np.floor(u[ok, 0]).astype(np.int64)
    return p


def pixel_size(window):
    return min((window.hi[k] - window.lo[k]) / window.npix[k] for k in range(2))


def error_stats(y_gpu, y_ref, window):
    """Per-ray source-position error |dy| (max over axes) in units of the pixel size."""
    pix = pixel_size(window)
    fin = np.isfinite(y_ref).all(1)
    err = np.abs(y_gpu[fin] - y_ref[fin]).max(1) / pix
    return {
        "n": int(err.size),
        "max": float(err.max()) if err.size else 0.0,
        "p50": float(np.median(err)) if err.size else 0.0,
        "p99": float(np.quantile(err, 0.99)) if err.size else 0.0,
        "frac_gt_1e-5": float((err > 1e-5).mean()) if err.size else 0.0,
    }


def abs_term_sum(field_spec, x):
    """sum_i m_i / |x - x_i| per ray (float64), the scale of a rigorous FP32 error bound."""
    L = field_spec.lens_xy.astype(np.float64)
    m = None if field_spec.masses is None else field_spec.masses.astype(np.float64)
    out = np.zeros(x.shape[0])
    for s in range(0, L.shape[0], 4096):
        d = x[:, None, :] - L[None, s:s + 4096, :]
        r = np.sqrt((d ** 2).sum(-1))
        t = 1.0 / r if m is None else m[None, s:s + 4096] / r
        out += t.sum(1)
    return out


U32 = 2.0 ** -24
# Worst-case relative error constants of the float32 body (units of u = 2^-24):
#   per term: d1/d2 rounding (1), d^2 and the fma forming r^2 (2), rcp.approx (<= 1 ulp: 2),
#   shared-reciprocal product and back-multiply (2), mass multiply (1)          -> 8
#   accumulation of a 64-lens group in float32: gamma_64 ~ 64                   -> 64
# The (hi, lo) TwoSum fold across groups is error-free; rs_trace's float64 epilogue adds ~1e-16.
K_TERM, K_GROUP = 8.0, 64.0


def per_ray_bound(field_spec, x, y_ref):
    """Rigorous bound on |y_gpu - y_exact| per ray for the float32 path."""
    B = abs_term_sum(field_spec, x)
    return (K_TERM + K_GROUP) * U32 * B + 1e-15 * (np.abs(y_ref).max(1) + np.abs(x).max(1))
