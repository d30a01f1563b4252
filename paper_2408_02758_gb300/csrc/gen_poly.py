"""Minimax polynomial coefficients for the float sine/cosine of the advection kernels.

Writes ``poly_coef.cuh``.  Method: the Remez exchange algorithm (E. Remez, 1934) on the
approximation of
  sin(pi r) = r * S(r^2)   and   cos(pi r) = C(r^2)   for |r| <= 1/4   (sinpi/cospi after
                                                                       reduction by 1/2)
  sin(r)    = r * S'(r^2)  and   cos(r)    = C'(r^2)  for |r| <= pi/4 (after reduction by pi/2)
minimising the absolute error of the value (what enters the velocity) with float-representable
coefficients; the exchange runs in float64 on a dense grid, and the final coefficients are
rounded to float32 and the achieved error is reported with float32 evaluation emulated.

It also writes the float-float tables of the re-advection kernel: (sin, cos)(pi j/64) for
j = -16..16 and (sin, cos)(j/32) for j = -26..26, each value split into a float pair h + l
(h = fl(v), l = fl(v - h)) from the double-precision value.

Run from the repository root:  python paper_2408_02758_gb300/csrc/gen_poly.py
"""
from __future__ import annotations

import math
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent


def remez(func, basis, a, b, n_iter=40, grid=400001):
    """Minimax (absolute error) fit of func on [a, b] by a combination of the basis functions."""
    m = len(basis)
    xs = np.linspace(a, b, grid)
    B = np.stack([phi(xs) for phi in basis], axis=1)
    fx = func(xs)
    k = np.arange(m + 1)
    ref = np.searchsorted(xs, 0.5 * (a + b) - 0.5 * (b - a) * np.cos(np.pi * k / m))
    ref = np.clip(ref, 0, grid - 1)
    coef = np.zeros(m)
    for _ in range(n_iter):
        A = np.concatenate([B[ref], ((-1.0) ** k)[:, None]], axis=1)
        sol = np.linalg.solve(A, fx[ref])
        coef, lev = sol[:m], sol[m]
        err = fx - B @ coef
        # one extremum per run of constant sign, then keep m + 1 alternating ones
        sgn = np.where(err >= 0, 1, -1)
        cut = np.flatnonzero(np.diff(sgn)) + 1
        seg = np.split(np.arange(grid), cut)
        ext = np.array([g[np.argmax(np.abs(err[g]))] for g in seg])
        while len(ext) > m + 1:
            ext = ext[1:] if abs(err[ext[0]]) < abs(err[ext[-1]]) else ext[:-1]
        if len(ext) < m + 1:
            break
        if np.array_equal(ext, ref):
            break
        ref = ext
    return coef


def fit_rounded(func, basis, a, b):
    """Minimax fit whose coefficients are float32: round the lowest-order coefficient, refit the
    others against the remaining error, and repeat (rounding each coefficient once)."""
    fixed = []
    for j in range(len(basis)):
        rest = basis[j:]

        def resid(z, fixed=tuple(fixed)):
            return func(z) - sum(c * phi(z) for c, phi in zip(fixed, basis))

        c = remez(resid, rest, a, b)
        fixed.append(float(np.float32(c[0])))
    return fixed


def fit_even_odd(fn_sin, fn_cos, half_width, n_sin, n_cos):
    """Fit in z = r^2 on [0, w^2]: sin = sqrt(z) * sum s_i z^i, cos = sum c_i z^i."""
    w2 = half_width ** 2
    sbasis = [lambda z, i=i: np.sqrt(z) * z ** i for i in range(n_sin)]
    cbasis = [lambda z, i=i: z ** i for i in range(n_cos)]
    s = fit_rounded(lambda z: fn_sin(np.sqrt(z)), sbasis, 0.0, w2)
    c = fit_rounded(lambda z: fn_cos(np.sqrt(z)), cbasis, 0.0, w2)
    return s, c, w2


def eval32(coefs, r, odd):
    """Horner in float32 on z = r*r, as the kernel evaluates it."""
    r = np.float32(r)
    z = (r * r).astype(np.float32)
    acc = np.full_like(z, np.float32(coefs[-1]))
    for cc in coefs[-2::-1]:
        acc = (acc * z + np.float32(cc)).astype(np.float32)
    if odd:
        acc = (acc * r).astype(np.float32)
    return acc


def main():
    out = []
    report = []
    for name, fs, fc, w, ns, nc in [
        ("PI", lambda x: np.sin(np.pi * x), lambda x: np.cos(np.pi * x), 0.25, 4, 5),
        ("RAD", np.sin, np.cos, math.pi / 4, 4, 5),
    ]:
        s, c, _ = fit_even_odd(fs, fc, w, ns, nc)
        s32 = [float(np.float32(v)) for v in s]
        c32 = [float(np.float32(v)) for v in c]
        r = np.linspace(-w, w, 400001, dtype=np.float64).astype(np.float32)
        es = np.abs(eval32(s32, r, True).astype(np.float64) - fs(r.astype(np.float64))).max()
        ec = np.abs(eval32(c32, r, False).astype(np.float64) - fc(r.astype(np.float64))).max()
        report.append(f"{name}: max |err| sin {es:.3e}, cos {ec:.3e} (float32 evaluation, |r| <= {w:.6f})")
        out.append(f"// {name}: sin = r * (s0 + z (s1 + ...)), cos = c0 + z (c1 + ...), z = r^2")
        out.append(f"constexpr float k{name}_S[{ns}] = {{" + ", ".join(f"{v:.9e}f" for v in s32) + "};")
        out.append(f"constexpr float k{name}_C[{nc}] = {{" + ", ".join(f"{v:.9e}f" for v in c32) + "};")
    def pair(v):
        h = np.float32(v)
        return float(h), float(np.float32(v - float(h)))

    rows = []
    for j in range(-26, 27):
        a = j / 32
        sh, sl = pair(math.sin(a))
        ch, cl = pair(math.cos(a))
        rows.append(f"  {{{sh:.9e}f, {sl:.9e}f, {ch:.9e}f, {cl:.9e}f}}")
    out.append("// float-float (sin, cos)(j / 32), j = -26..26: {sin_h, sin_l, cos_h, cos_l}")
    out.append("__device__ __align__(16) const float kDS_SIN_TAB[53][4] = {\n" + ",\n".join(rows) + "};")
    # one period of sin/cos(pi x) at spacing 1/512, from 50-digit values rounded to float-float
    import mpmath

    mpmath.mp.dps = 50

    def pair_mp(v):
        h = np.float32(float(v))
        return float(h), float(np.float32(float(v - mpmath.mpf(float(h)))))

    rows = []
    for j in range(-512, 513):
        sh, sl = pair_mp(mpmath.sinpi(mpmath.mpf(j) / 512))
        ch, cl = pair_mp(mpmath.cospi(mpmath.mpf(j) / 512))
        rows.append(f"  {{{sh:.9e}f, {sl:.9e}f, {ch:.9e}f, {cl:.9e}f}}")
    out.append("// float-float (sin, cos)(pi j / 512), j = -512..512: {sin_h, sin_l, cos_h, cos_l}")
    out.append("__device__ __align__(16) const float kDS_SINPI512_TAB[1025][4] = {\n" + ",\n".join(rows) + "};")
    text = ("// Generated by gen_poly.py (Remez exchange, float32 coefficients); do not edit by hand.\n"
            "// " + "\n// ".join(report) + "\n#pragma once\n\nnamespace ftle {\n" + "\n".join(out) + "\n}  // namespace ftle\n")
    (HERE / "poly_coef.cuh").write_text(text)
    print("\n".join(report))


if __name__ == "__main__":
    main()
