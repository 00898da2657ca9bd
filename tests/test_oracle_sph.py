"""Pins of the oracle's SPH kernel, density, pressure force and LJ force."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2602_19873_gb300 import workloads as wl


def test_kernel_normalisation_and_shape(orc):
    # 4 pi int_0^{2h} r^2 W(r,h) dr = 1 for any h
    for h in (0.37, 1.0, 2.5):
        v, err = integrate.quad(lambda r: 4 * math.pi * r * r * orc.W(r, h), 0, 2 * h,
                                points=[h], epsabs=1e-14, epsrel=1e-13)
        assert abs(v - 1.0) < 1e-12
    assert orc.W(0.0, 1.0) == pytest.approx(1.0 / math.pi, rel=1e-15)
    assert orc.w(2.0) == 0.0 and orc.w(2.5) == 0.0
    # C^2 continuity at q = 1 and q = 2, and w' is the derivative of w
    e = 1e-7
    for q in (1.0, 2.0):
        assert abs(orc.w(q - e) - orc.w(q + e)) < 1e-6
        assert abs(orc.dw(q - e) - orc.dw(q + e)) < 1e-6
        d2l = (orc.dw(q - e) - orc.dw(q - 3 * e)) / (2 * e)
        d2r = (orc.dw(q + 3 * e) - orc.dw(q + e)) / (2 * e) if q < 2 else 0.0
        assert abs(d2l - d2r) < 1e-4
    for q in np.linspace(0.01, 1.99, 37):
        fd = (orc.w(q + 1e-6) - orc.w(q - 1e-6)) / 2e-6
        assert abs(fd - orc.dw(q)) < 1e-7


def _sorted(orc, d):
    k = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    p = orc.sort(k)
    return [np.asarray(d[a])[p] for a in ("x", "y", "z", "h", "m")]


def test_fp32_predicate_agrees_with_exact_distance(orc):
    """The FP32 set differs from the exact FP64 set only at the boundary
    (|d - r| within a few ulps), so a dropped term or sign shows here."""
    d = wl.plummer(3000, n_spheres=2, seed=31, n_target=50)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    P = np.stack([xs, ys, zs], 1).astype(np.float64)
    for i in range(0, len(xs), 37):
        r = 2.0 * float(hs[i])
        dist = np.linalg.norm(P - P[i], axis=1)
        exact = set(np.nonzero(dist < r)[0].tolist()) - {i}
        got = set(g_idx[g_off[i]:g_off[i + 1]].tolist())
        for j in exact ^ got:
            assert abs(dist[j] - r) <= 1e-6 * r


def test_density_against_direct_sum(orc):
    d = wl.evrard(2500, seed=32, n_target=50)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    rho = orc.density(xs, ys, zs, hs, ms, d["box"], g_off, g_idx, np.arange(len(xs)))
    P = np.stack([xs, ys, zs], 1).astype(np.float64)
    for i in range(0, len(xs), 41):
        h = float(hs[i])
        q = np.linalg.norm(P - P[i], axis=1) / h
        w = np.where(q < 1, 1 - 1.5 * q ** 2 + 0.75 * q ** 3, np.where(q < 2, 0.25 * (2 - q) ** 3, 0))
        want = float(np.sum(ms.astype(np.float64) * w) / (math.pi * h ** 3))
        assert rho[i] == pytest.approx(want, rel=1e-9)


def test_density_of_uniform_cube_is_one(orc):
    d = wl.uniform(30000, seed=33, n_target=100.0)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    rho = orc.density(xs, ys, zs, hs, ms, d["box"], g_off, g_idx, np.arange(len(xs)))
    # Poisson points: E[sum over the others] = (n-1)/n; the self term adds
    # m W(0,h) = 1/(n pi h^3) on top
    n, h = len(xs), float(hs[0])
    want = (n - 1) / n + 1.0 / (n * math.pi * h ** 3)
    assert abs(rho.mean() - want) < 0.003


def _energy(orc, xs, ys, zs, hs, ms, box, K, gamma):
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, box, 2.0)
    rho = orc.density(xs, ys, zs, hs, ms, box, g_off, g_idx, np.arange(len(xs)))
    return float(np.sum(ms.astype(np.float64) * K * rho ** (gamma - 1) / (gamma - 1))), rho


def test_pressure_force_is_minus_energy_gradient(orc):
    """With fixed h_i and P = K rho^gamma, the symmetric pressure force equals
    -(1/m_k) dE/dx_k for E = sum_i m_i K rho_i^(gamma-1)/(gamma-1)."""
    rng = np.random.default_rng(34)
    n = 300
    d = {"x": rng.normal(0, 0.3, n).astype(np.float32), "y": rng.normal(0, 0.3, n).astype(np.float32),
         "z": rng.normal(0, 0.3, n).astype(np.float32), "kind": 1,
         "h": (0.15 + 0.1 * rng.random(n)).astype(np.float32),
         "m": (1.0 + rng.random(n)).astype(np.float32) / n,
         "box": {"lo": np.full(3, -3, np.float32), "hi": np.full(3, 3, np.float32),
                 "periodic": np.zeros(3, np.int32)}}
    xs, ys, zs, hs, ms = _sorted(orc, d)
    K, gamma = 0.7, 5.0 / 3.0
    E0, rho = _energy(orc, xs, ys, zs, hs, ms, d["box"], K, gamma)
    pres = K * rho ** gamma
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 2.0)
    p_off, p_idx = orc.symmetrize(g_off, g_idx)
    ax, ay, az, _ = orc.sph_force(xs, ys, zs, hs, ms, rho, pres, d["box"], p_off, p_idx, np.arange(n))
    acc = np.stack([ax, ay, az], 1)
    # momentum conservation
    assert np.abs((ms[:, None].astype(np.float64) * acc).sum(0)).max() < 1e-12 * np.abs(
        ms[:, None] * acc).sum()
    center = np.argsort(np.linalg.norm(np.stack([xs, ys, zs], 1), axis=1))[:6]
    for k in center:
        for a, arr in enumerate((xs, ys, zs)):
            step = 1e-4 * float(hs[k])
            vals = []
            for sgn in (+1, -1):
                pert = [xs.copy(), ys.copy(), zs.copy()]
                pert[a][k] = np.float32(float(arr[k]) + sgn * step)
                vals.append((_energy(orc, *pert, hs, ms, d["box"], K, gamma)[0], float(pert[a][k])))
            grad = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            want = -grad / float(ms[k])
            assert acc[k, a] == pytest.approx(want, rel=2e-4, abs=1e-6 * np.abs(acc).max())


def test_lj_force_energy_and_newton3(orc):
    d = wl.lj_fluid(1500, seed=35)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    box, eps, sig = d["box"], 1.0, 0.3
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, box, 1.0)
    n = len(xs)
    fx, fy, fz, fa = orc.lj_force(xs, ys, zs, box, eps, sig, g_off, g_idx, np.arange(n))
    F = np.stack([fx, fy, fz], 1)
    assert np.abs(F.sum(0)).max() < 1e-10 * np.abs(F).sum()
    # energy against a direct double loop
    P = np.stack([xs, ys, zs], 1).astype(np.float64)
    L = float(box["hi"][0] - box["lo"][0])
    E = 0.0
    for i in range(n):
        dv = P - P[i]
        dv -= L * np.round(dv / L)
        r2 = (dv ** 2).sum(1)
        sel = (np.arange(n) > i) & (r2 < 0.81)
        sr6 = (sig * sig / r2[sel]) ** 3
        E += float(np.sum(4 * eps * (sr6 * sr6 - sr6)))
    assert orc.lj_energy(xs, ys, zs, box, eps, sig, g_off, g_idx) == pytest.approx(E, rel=1e-10)
    # F = -dE/dx on a few particles (pairs never cross the cutoff here)
    for k in (3, n // 2):
        for a, arr in enumerate((xs, ys, zs)):
            vals = []
            for sgn in (+1, -1):
                pert = [xs.copy(), ys.copy(), zs.copy()]
                pert[a][k] = np.float32(float(arr[k]) + sgn * 1e-4)
                go, gi = orc.gather_all(*pert, hs, box, 1.0)
                vals.append((orc.lj_energy(*pert, box, eps, sig, go, gi), float(pert[a][k])))
            grad = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            if abs(grad) > 1e3 * abs(F[k, a]) + 1e3:
                continue  # a pair crossed rc inside the step (energy jump)
            assert F[k, a] == pytest.approx(-grad, rel=1e-3, abs=1e-3)
