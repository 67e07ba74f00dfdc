"""FP64 oracle of the image-quality metric reported beside PSNR: SSIM of the
affiliated eye against its full render (Table 2 reports SSIM; this is the
structural similarity of Wang et al. 2004 in the convention of the 2DGS/3DGS
evaluation code the paper's numbers come from).

TEST INFRASTRUCTURE ONLY: imported by tests/ and bench.py's CPU baseline, never
by the product. Plain numpy/scipy in float64:

  window   11 x 11 Gaussian, sigma 1.5, normalised to sum 1
  filter   same-size 2-D convolution of each channel with zero padding (the
           window is symmetric, so convolution and correlation agree)
  maps     mu_x = w * x, mu_y = w * y, s_xx = w * x^2 - mu_x^2,
           s_yy = w * y^2 - mu_y^2, s_xy = w * (x y) - mu_x mu_y
  SSIM     (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2))
           with C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1), averaged over every
           pixel of every channel

Reading (the paper names SSIM without its constants): the window, constants and
zero padding of the 2DGS/3DGS evaluation code. Pins: tests/test_oracle_metrics.py
(identity, a brute-force window sum, constant images in closed form, symmetry).
"""
import numpy as np
from scipy import signal

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> np.ndarray:
    """size x size Gaussian weights, normalised to sum 1 (outer product of the
    normalised 1-D window)."""
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-(x ** 2) / (2.0 * sigma ** 2))
    g /= g.sum()
    return np.outer(g, g)


def _filter(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    return signal.convolve2d(img, w, mode="same", boundary="fill", fillvalue=0.0)


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel SSIM of two single-channel images [H, W]."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = gaussian_window()
    mx, my = _filter(x, w), _filter(y, w)
    sxx = _filter(x * x, w) - mx * mx
    syy = _filter(y * y, w) - my * my
    sxy = _filter(x * y, w) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(a: np.ndarray, b: np.ndarray) -> float:
    """Mean SSIM of two images [C, H, W] (or [H, W]) over pixels and channels."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.ndim == 2:
        return float(ssim_map(a, b).mean())
    return float(np.mean([ssim_map(a[c], b[c]) for c in range(a.shape[0])]))
