"""Calibrates the 2-D steady approximate mobility of App. B (Eq.
fg_steady_2d) for the library's kernels, following the paper's procedure
(Sec. IV.B, App. B): the pair mobility of two markers is measured in a
periodic unit square, normalised as

  f~(x) = -(4 pi eta) (f(x) - f(0)),   g~(x) = (4 pi eta) g(x),   x = r / h,

(M_ij = f(r) I + g(r) r^ r^T), and the rational forms

  f~(x) = (a0 x^2 + a1 x^3 + a2 x^3 ln x) / (1 + a3 x + a4 x^2 + a2 x^3)
  g~(x) = (b0 x^2 + b1 x^3) / (1 + b2 x + b3 x^2 + b1 x^3)

are fitted by least squares; the marker radius a follows from the self
mobility f(0) = (4 pi eta)^-1 ln(l / (3.708 a)).  The paper does not print
its coefficients; this script produces the library's.

The pair mobility is the grid's own: the library's tabulated pair mobility
(IBR_MOB_PAIR: exact-to-1e-9 Stokes solves of point forces at two sub-cell
source positions, averaged), read back through ibr_op_mtilde for markers
placed at many distances and directions.  Needs a GPU.

Usage: python -m paper_1505_07865_gb300.fit_mobility_2d [--out file.json]
"""
import argparse
import json
import os
import sys

import numpy as np
from scipy.optimize import least_squares

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_1505_07865_gb300 import abi  # noqa: E402


def pair_mobility_samples(kernel, n=256, N=360, xmax=20.0, seed=5):
    """(x, f, g) samples and the self-mobility f(0) on an n^2 periodic unit
    square (eta = 1) from the library's pair-mobility M~."""
    import torch

    h = 1.0 / n
    rng = np.random.default_rng(seed)
    c = np.array([0.5, 0.5]) + rng.uniform(-0.5, 0.5, 2) * h
    xs = np.exp(rng.uniform(np.log(0.2), np.log(xmax), N - 1))
    th = rng.uniform(0, 2 * np.pi, N - 1)
    rel = np.concatenate([np.zeros((1, 2)), (xs * h)[:, None] * np.stack([np.cos(th), np.sin(th)], 1)])
    G = abi.create_grid(2, (n, n), (1.0, 1.0), kernel=kernel, precision=abi.FP64)
    try:
        abi.add_body(G, c)
        abi.set_markers(G, 0, rel)
        o = abi.solve_opts_default()
        o.mob_model = abi.MOB_PAIR
        abi.prepare(G, o)
        out = torch.zeros((2 * N) ** 2, dtype=torch.float64, device="cuda")
        abi.op_mtilde(G, 0, out)
        M = out.cpu().numpy().reshape(2 * N, 2 * N)
    finally:
        abi.destroy_grid(G)
    f0 = float(np.mean([0.5 * (M[2 * i, 2 * i] + M[2 * i + 1, 2 * i + 1]) for i in range(N)]))
    X, F, Gg = [], [], []
    for i in range(N):
        for j in range(i + 1, N):
            d = (rel[i] - rel[j]) / h
            x = float(np.hypot(*d))
            if x > xmax or x < 0.1:
                continue
            e = d / x
            p = np.array([-e[1], e[0]])
            B = M[2 * i:2 * i + 2, 2 * j:2 * j + 2]
            f = float(p @ B @ p)
            X.append(x)
            F.append(f)
            Gg.append(float(e @ B @ e) - f)
    return np.array(X), np.array(F), np.array(Gg), f0


def f_form(a, x):
    return (a[0] * x ** 2 + a[1] * x ** 3 + a[2] * x ** 3 * np.log(x)) / (1 + a[3] * x + a[4] * x ** 2 + a[2] * x ** 3)


def g_form(b, x):
    return (b[0] * x ** 2 + b[1] * x ** 3) / (1 + b[2] * x + b[3] * x ** 2 + b[1] * x ** 3)


def fit(kernel, n=256):
    X, F, Gg, f0 = pair_mobility_samples(kernel, n)
    eta = 1.0
    ft = -(4 * np.pi * eta) * (F - f0)
    gt = (4 * np.pi * eta) * Gg
    ra = least_squares(lambda a: f_form(a, X) - ft, [0.6, 0.3, 1.0, 0.1, 0.6], bounds=([0, -5, 1e-3, 0, 0], 10))
    rb = least_squares(lambda b: g_form(b, X) - gt, [0.25, 1.0, 0.1, 0.5], bounds=([0, 1e-3, 0, 0], 10))
    aoh = 1.0 / (3.708 * np.exp(4 * np.pi * eta * f0)) / (1.0 / n)
    return {"kernel": int(kernel), "n": n, "samples": int(X.size), "f0": f0, "a_over_h": float(aoh),
            "a": [float(v) for v in ra.x], "b": [float(v) for v in rb.x],
            "rms_f": float(np.sqrt(np.mean(ra.fun ** 2))), "rms_g": float(np.sqrt(np.mean(rb.fun ** 2))),
            "max_f": float(np.abs(ra.fun).max()), "max_g": float(np.abs(rb.fun).max())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    res = {"procedure": "App. B / Sec. IV.B fits of the library's own periodic pair mobility (IBR_MOB_PAIR), "
                        "unit square, eta = 1", "fits": []}
    for kernel in (abi.KERNEL_PESKIN4, abi.KERNEL_BKP6):
        for n in (128, 256):
            r = fit(kernel, n)
            res["fits"].append(r)
            print(json.dumps(r), flush=True)
    if args.out:
        json.dump(res, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
