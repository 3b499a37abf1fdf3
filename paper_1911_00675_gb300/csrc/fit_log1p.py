"""Fits the polynomial of log1p_reduced (pmh_device.cuh): r(f) = (log1p(f) - f) / f^2 on
[sqrt(1/2) - 1, sqrt(2) - 1] by least squares on Chebyshev nodes, weighted for the relative error
of f + f^2 r(f), and reports the worst relative error of its FP32 evaluation against FP64 log1p.
The device code holds the degree-8 coefficients this prints (rounded to FP32).

    python paper_1911_00675_gb300/csrc/fit_log1p.py
"""
import numpy as np


def fit(deg, nodes=4000):
    a, b = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    t = np.cos(np.pi * (np.arange(nodes) + 0.5) / nodes)
    f = (a + b) / 2 + (b - a) / 2 * t
    f = f[np.abs(f) > 1e-6]
    target = (np.log1p(f) - f) / f**2
    wgt = f**2 / np.abs(np.log1p(f))
    V = np.vander(f, deg + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(V * wgt[:, None], target * wgt, rcond=None)
    return coef.astype(np.float32)


def worst_rel_error(c32, points=2_000_001):
    a, b = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    fg = np.linspace(a, b, points).astype(np.float32)
    fg = fg[fg != 0]
    r = np.float32(c32[-1])
    for cc in c32[-2::-1]:
        r = (r * fg + np.float32(cc)).astype(np.float32)   # two roundings per step: pessimistic vs FMA
    val = (fg + (fg * fg).astype(np.float32) * r).astype(np.float32)
    ref = np.log1p(fg.astype(np.float64))
    return float((np.abs(val.astype(np.float64) - ref) / np.abs(ref)).max())


if __name__ == "__main__":
    c = fit(8)
    print("coefficients (r_0 .. r_8):", [float(x) for x in c])
    print("worst relative error: %.3g (%.2f ulp of 2^-24)" % (worst_rel_error(c), worst_rel_error(c) / 2**-24))
