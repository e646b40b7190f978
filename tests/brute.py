"""Brute-force nearest-source search (Sec. 3, the naive approach: every pixel
against every source pixel).  Independent of the oracle; tiny inputs only."""
import numpy as np

INF32 = np.iinfo(np.int32).max


def sources(mask, mode):
    m = np.asarray(mask) != 0
    return m if mode == 0 else ~m


def brute_edt(mask, mode=0):
    """Squared distance to the nearest source pixel (INT32_MAX if none)."""
    src = sources(mask, mode)
    shape = src.shape
    coords = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), -1).reshape(-1, len(shape))
    s = coords[src.reshape(-1)]
    if s.shape[0] == 0:
        return np.full(shape, INF32, dtype=np.int64)
    d = ((coords[:, None, :] - s[None, :, :]) ** 2).sum(-1)
    return d.min(1).reshape(shape)


def brute_edt_many(masks, mode=0):
    """Vectorised over a stack of equally shaped 2-D masks [n, H, W]."""
    masks = np.asarray(masks)
    n, H, W = masks.shape
    src = (masks != 0) if mode == 0 else (masks == 0)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    p = np.stack([yy.reshape(-1), xx.reshape(-1)], -1)
    d2 = ((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)  # [P, Q]
    big = np.iinfo(np.int64).max // 4
    flat = src.reshape(n, -1)
    cand = np.where(flat[:, None, :], d2[None, :, :], big)
    out = cand.min(-1)
    out[out >= big] = INF32
    return out.reshape(n, H, W)


def feature_valid(mask, mode, D, F):
    """True when every F(p) is a source and |p - F(p)|^2 == D(p)."""
    src = sources(mask, mode)
    shape = src.shape
    flat_src = src.reshape(-1)
    Fr = F.reshape(-1)
    Dr = D.reshape(-1).astype(np.int64)
    none = Dr == INF32
    if np.any(Fr[none] != -1):
        return False
    ok = ~none
    if not np.all((Fr[ok] >= 0) & (Fr[ok] < flat_src.size)):
        return False
    if not np.all(flat_src[Fr[ok]]):
        return False
    p = np.stack(np.unravel_index(np.arange(Fr.size)[ok], shape), -1)
    q = np.stack(np.unravel_index(Fr[ok], shape), -1)
    return bool(np.all(((p - q) ** 2).sum(-1) == Dr[ok]))
