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


def _pair_system(p1, p2, box=None):
    xs, ys, zs = (np.array([p1[a], p2[a]], np.float32) for a in range(3))
    if box is None:
        box = {"lo": np.full(3, -10, np.float32), "hi": np.full(3, 10, np.float32),
               "periodic": np.zeros(3, np.int32)}
    off = np.array([0, 1, 2], np.int64)
    idx = np.array([1, 0], np.int64)
    return xs, ys, zs, box, off, idx


def test_ljc_two_particles_closed_forms(orc):
    """Coulomb's law and the LJ minimum for one pair (Sec. III-B interactions)."""
    xs, ys, zs, box, off, idx = _pair_system((0.1, -0.2, 0.3), (0.5, 0.1, -0.3))
    P = np.stack([xs, ys, zs], 1).astype(np.float64)
    u = P[0] - P[1]
    r = float(np.linalg.norm(u))
    q = np.array([2.0, -0.5], np.float32)
    kc = 1.5
    # Coulomb only: |F| = kc q1 q2 / r^2 along the unit vector from 2 to 1
    fx, fy, fz, fa = orc.ljc_force(xs, ys, zs, box, 0.0, 0.3, q, kc, off, idx, [0, 1])
    want = kc * 2.0 * -0.5 / r ** 2 * (u / r)
    assert np.allclose([fx[0], fy[0], fz[0]], want, rtol=1e-12, atol=0)
    assert np.allclose([fx[1], fy[1], fz[1]], -want, rtol=1e-12, atol=0)
    assert fa[0] == pytest.approx(abs(kc * 2.0 * -0.5) / r ** 2, rel=1e-12)
    assert orc.ljc_energy(xs, ys, zs, box, 0.0, 0.3, q, kc, off, idx) == pytest.approx(
        kc * 2.0 * -0.5 / r, rel=1e-12)
    # LJ only at the potential minimum r = 2^(1/6) sigma: zero force, E = -eps
    sig = r / 2 ** (1 / 6)
    fx, fy, fz, _ = orc.ljc_force(xs, ys, zs, box, 0.8, sig, None, kc, off, idx, [0, 1])
    assert max(abs(fx[0]), abs(fy[0]), abs(fz[0])) < 1e-12
    assert orc.ljc_energy(xs, ys, zs, box, 0.8, sig, None, kc, off, idx) == pytest.approx(-0.8, rel=1e-12)
    # repulsive inside the minimum: the force on 1 points away from 2
    fx, fy, fz, _ = orc.ljc_force(xs, ys, zs, box, 0.8, 1.1 * sig, None, kc, off, idx, [0, 1])
    assert float(np.dot([fx[0], fy[0], fz[0]], u)) > 0


def test_ljc_periodic_minimum_image(orc):
    """A pair straddling a periodic face interacts across it (distance 0.2,
    not 0.8)."""
    box = {"lo": np.zeros(3, np.float32), "hi": np.ones(3, np.float32),
           "periodic": np.ones(3, np.int32)}
    xs, ys, zs, box, off, idx = _pair_system((0.05, 0.5, 0.5), (0.85, 0.5, 0.5), box)
    q = np.array([1.0, 1.0], np.float32)
    fx, fy, fz, _ = orc.ljc_force(xs, ys, zs, box, 0.0, 0.3, q, 1.0, off, idx, [0, 1])
    r = float(np.float32(1.0) - (np.float32(0.85) - np.float32(0.05)))
    # like charges repel: particle 0 is pushed in +x (away from its image at -0.15)
    assert fx[0] == pytest.approx(1.0 / r ** 2, rel=1e-6)
    assert abs(fy[0]) < 1e-12 and abs(fz[0]) < 1e-12


def test_ljc_reduces_to_lj_without_charges(orc):
    d = wl.lj_fluid(800, seed=36)
    xs, ys, zs, hs, ms = _sorted(orc, d)
    g_off, g_idx = orc.gather_all(xs, ys, zs, hs, d["box"], 1.0)
    rows = np.arange(len(xs))
    a = orc.lj_force(xs, ys, zs, d["box"], 1.0, 0.3, g_off, g_idx, rows)
    b = orc.ljc_force(xs, ys, zs, d["box"], 1.0, 0.3, None, 138.9, g_off, g_idx, rows)
    c = orc.ljc_force(xs, ys, zs, d["box"], 1.0, 0.3, np.zeros(len(xs), np.float32), 138.9,
                      g_off, g_idx, rows)
    for u, v, w in zip(a, b, c):
        assert np.array_equal(u, v) and np.array_equal(u, w)


def test_ljc_force_is_minus_energy_gradient(orc):
    """Newton III and F = -dE/dx for LJ + Coulomb at the interaction cutoff of
    the Verlet-buffer workload (pairs that cross rc inside the step skipped)."""
    d = wl.lj_coulomb(1500, seed=37)
    k_ = orc.keys(d["x"], d["y"], d["z"], d["box"], d["kind"])
    p = orc.sort(k_)
    xs, ys, zs, q = (np.asarray(d[a])[p] for a in ("x", "y", "z", "q"))
    box, rc, kc = d["box"], d["rc"], d["kc"]
    hr = np.full(len(xs), np.float32(rc))
    g_off, g_idx = orc.gather_all(xs, ys, zs, hr, box, 1.0)
    n = len(xs)
    fx, fy, fz, fa = orc.ljc_force(xs, ys, zs, box, 1.0, 0.3, q, kc, g_off, g_idx, np.arange(n))
    F = np.stack([fx, fy, fz], 1)
    assert np.abs(F.sum(0)).max() < 1e-10 * np.abs(F).sum()
    assert abs(float(q.astype(np.float64).sum())) <= 1.0
    checked = 0
    for k in (5, n // 3, n - 7):
        for a, arr in enumerate((xs, ys, zs)):
            vals = []
            for sgn in (+1, -1):
                pert = [xs.copy(), ys.copy(), zs.copy()]
                pert[a][k] = np.float32(float(arr[k]) + sgn * 1e-4)
                go, gi = orc.gather_all(*pert, hr, box, 1.0)
                if not (np.array_equal(go, g_off) and np.array_equal(gi, g_idx)):
                    vals = None  # the pair set changed inside the step (energy jump)
                    break
                vals.append((orc.ljc_energy(*pert, box, 1.0, 0.3, q, kc, go, gi), float(pert[a][k])))
            if vals is None:
                continue
            grad = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            assert F[k, a] == pytest.approx(-grad, rel=1e-3, abs=1e-6 * np.abs(F).max())
            checked += 1
    assert checked >= 6
