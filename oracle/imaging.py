"""Plain CPU oracle of the imaging half of the major cycle (Sec. 2.2 and the
Cotton-Schwab steps that follow Eq. 6): gridding and FFT to a dirty image,
Hogbom clean (Eqs. 4-6), and the loop of major cycles around the model
prediction.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import it; the
CUDA library never calls it and shares no code with it. numpy only.

Readings taken where the paper is silent (listed with the others in the
design notes):
  I1  Gridding: nearest cell (no convolution kernel), every visibility and
      its Hermitian conjugate at -B, unit weights; a visibility whose cell or
      mirrored cell falls outside the grid is left out. The w term is
      ignored in imaging (the 2-D transform of Eq. 2); the prediction keeps
      it.
  I2  Geometry: an n x n image (n even) of pixel size dl (radians), pixel
      (ix, iy) at l = (ix - n/2) dl, m = (iy - n/2) dl; uv cell size
      du = 1 / (n dl), cell (iu, iv) at u = (iu - n/2) du, v = (iv - n/2) du;
      arrays are indexed [iy][ix] and [iv][iu].
  I3  Dirty image I(l, m) = (1/W) sum over cells of G(u, v)
      exp(-i 2 pi (u l + v m)), real part, W = number of gridded entries
      (both half-planes): a point source of flux C at the phase centre gives
      I = C there, and the beam (PSF, the image of unit visibilities) is 1 at
      its centre.
  I4  Hogbom: "the pixel with the maximum value" is taken literally (the
      largest value, not the largest magnitude); ties go to the first pixel
      in row-major order. The beam is centred at pixel (n/2, n/2) and is
      subtracted wherever its shifted copy overlaps the image. The clean
      stops after max_iter iterations or when the maximum falls below the
      threshold. The arithmetic is float32 (the precision the GPU decides
      the argmax in): the component flux fl(g C), the update
      fl(I - fl(f B)).
  I5  The w-corrected dirty image (what w-projection gridding, Sec. 3.6.2's
      wide-field imaging, approximates): I3 with each entry's exponent
      carrying w (n(l, m) - 1), evaluated as a direct sum over the
      visibilities (every visibility inside the grid, so W = 2 N).
"""
from __future__ import annotations

import numpy as np


def grid_nn(uvw, vis, n, dl):
    """Nearest-cell gridding (I1, I2): complex grid [n][n] and the number of
    gridded entries W."""
    uvw = np.asarray(uvw, dtype=np.float64)
    vis = np.asarray(vis, dtype=np.complex128)
    inv_du = n * dl                                   # 1 / du
    G = np.zeros((n, n), dtype=np.complex128)
    W = 0
    for (u, v, _), V in zip(uvw, vis):
        ru, rv = np.rint(u * inv_du), np.rint(v * inv_du)
        if not (-n // 2 < ru < n // 2 and -n // 2 < rv < n // 2):
            continue
        iu, iv = int(ru) + n // 2, int(rv) + n // 2
        ju, jv = n // 2 - int(ru), n // 2 - int(rv)
        G[iv, iu] += V
        G[jv, ju] += np.conj(V)
        W += 2
    return G, W


def image_from_grid(G, W):
    """Dirty image of a grid (I3), by the FFT: the index shifts put u = 0 and
    l = 0 at n/2."""
    if W == 0:
        return np.zeros(G.shape)
    F = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(G)))
    return F.real / W


def image_from_grid_direct(G, W, dl):
    """The same image by its definition, the double sum over cells (I3); for
    small grids only."""
    n = G.shape[0]
    du = 1.0 / (n * dl)
    ax = (np.arange(n) - n // 2)
    u = ax * du
    l = ax * dl
    E = np.exp(-2j * np.pi * np.outer(u, l))          # [cell, pixel] along one axis
    # I[iy][ix] = sum_{iv,iu} G[iv][iu] E[iv][iy] E[iu][ix]
    return (E.T @ G @ E).real / W if W else np.zeros((n, n))


def dirty_image(uvw, vis, n, dl):
    G, W = grid_nn(uvw, vis, n, dl)
    return image_from_grid(G, W)


def dirty_beam(uvw, n, dl):
    """The PSF: the dirty image of unit visibilities."""
    return dirty_image(uvw, np.ones(len(uvw), dtype=np.complex128), n, dl)


def dirty_image_exact(uvw, vis, n, dl, ix, iy):
    """The w-corrected dirty image at pixels (ix, iy) by its definition
    (reading I5): the direct sum over the visibilities and their Hermitian
    conjugates of V exp(-i 2 pi (u l + v m + w (n(l, m) - 1))), real part,
    over W = 2 N entries, n(l, m) = sqrt(1 - l^2 - m^2): the image w-
    projection gridding approximates. A point source of flux C observed as
    V = C exp(i 2 pi B.(l0, m0, n0 - 1)) gives I = C at (l0, m0) for any w."""
    uvw = np.asarray(uvw, dtype=np.float64)
    vis = np.asarray(vis, dtype=np.complex128)
    ix = np.atleast_1d(np.asarray(ix))
    iy = np.atleast_1d(np.asarray(iy))
    l = (ix - n // 2) * dl
    m = (iy - n // 2) * dl
    r2 = l * l + m * m
    nm1 = -r2 / (1.0 + np.sqrt(1.0 - r2))             # n - 1 without cancellation
    s = np.stack([l, m, nm1], axis=1)                 # [pixel][3]
    out = np.zeros(len(l))
    for k0 in range(0, len(uvw), 4096):               # chunks of visibilities
        ph = uvw[k0:k0 + 4096] @ s.T                  # [vis][pixel]
        out += (vis[k0:k0 + 4096, None] * np.exp(-2j * np.pi * ph)).real.sum(axis=0)
    return out / len(uvw) if len(uvw) else out


def hogbom(image, psf, gain, max_iter, threshold):
    """Hogbom clean (Eq. 4), float32 throughout (I4). Returns the residual
    image, the component pixels (row-major index iy n + ix) and fluxes
    g C_n (Eq. 5)."""
    img = np.array(image, dtype=np.float32, copy=True)
    B = np.asarray(psf, dtype=np.float32)
    n = img.shape[0]
    c = n // 2
    g = np.float32(gain)
    pix, flux = [], []
    for _ in range(max_iter):
        p = int(np.argmax(img))
        py, px = divmod(p, n)
        peak = img[py, px]
        if peak < np.float32(threshold):
            break
        f = np.float32(g * peak)
        # image pixel q overlaps beam pixel q - p + c
        y0, y1 = max(0, py - c), min(n, py - c + n)
        x0, x1 = max(0, px - c), min(n, px - c + n)
        sub = B[y0 - py + c:y1 - py + c, x0 - px + c:x1 - px + c]
        img[y0:y1, x0:x1] = img[y0:y1, x0:x1] - np.float32(f) * sub
        pix.append(p)
        flux.append(f)
    return img, np.array(pix, dtype=np.int64), np.array(flux, dtype=np.float32)


def pixel_lm(pix, n, dl):
    """(l, m) of row-major pixel indices (I2)."""
    py, px = np.divmod(np.asarray(pix, dtype=np.int64), n)
    return (px - n // 2) * dl, (py - n // 2) * dl


def major_cycles(uvw, vis_obs, n, dl, gain, minor_iter, threshold, n_major, predict):
    """Cotton-Schwab major cycles (the steps after Eq. 6) with the model
    visibilities from ``predict(l, m, flux, uvw)`` (Eq. 12 or Eq. 17):
    dirty image of the residuals, Hogbom minor cycles, prediction from every
    component found so far, subtraction; ends after n_major cycles or a
    cycle without components. Returns the component lists (pixels, fluxes),
    the residual visibilities and the dirty image of the final residual
    visibilities."""
    psf = dirty_beam(uvw, n, dl)
    resid = np.asarray(vis_obs, dtype=np.complex128).copy()
    pix_all, flux_all = [], []
    for _ in range(n_major):
        dirty = dirty_image(uvw, resid, n, dl)
        _, pix, flux = hogbom(dirty, psf, gain, minor_iter, threshold)
        if len(pix) == 0:
            break
        pix_all.extend(pix.tolist())
        flux_all.extend(flux.tolist())
        l, m = pixel_lm(pix_all, n, dl)
        resid = np.asarray(vis_obs) - predict(l, m, np.asarray(flux_all, dtype=np.float64), uvw)
    img = dirty_image(uvw, resid, n, dl)
    return np.array(pix_all, dtype=np.int64), np.array(flux_all, dtype=np.float32), resid, img
