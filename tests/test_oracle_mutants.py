"""The oracle's pins catch plausible mistakes: each mutant below plants one (a dropped term, a
wrong sign, index or constant, a transposed operand) in a copy of the oracle, and the pin tests
that cover that part, run on the copy, must fail.  The copies live in a temporary directory; the
oracle itself is never modified.  The mutants run as parallel subprocesses."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle", "ns_oracle.py")

CORE = ["tests/test_oracle_tridiag.py", "tests/test_oracle_ops.py", "tests/test_oracle_step.py"]
BL = ["tests/test_oracle_bl.py"]
CFL = ["tests/test_oracle_cfl.py"]
RCY = ["tests/test_oracle_recycle.py"]

# name: (text in the oracle, replacement, pin files)
MUTANTS = {
    # RK3, interpolation, stencils, grid metrics
    "zeta_sign": ("RK3_ZETA = (0.0, -17.0 / 60.0, -5.0 / 12.0)", "RK3_ZETA = (0.0, 17.0 / 60.0, -5.0 / 12.0)", CORE),
    "gamma_value": ("RK3_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)", "RK3_GAMMA = (8.0 / 15.0, 5.0 / 12.0, 2.0 / 3.0)", CORE),
    "interp_swap": ("wlo = 1.0 - whi ", "wlo = whi; whi = 1.0 - wlo ", CORE),
    "wall_hm": ("hm[0] = g.yc[0] - g.yf[0]", "hm[0] = g.hc[0]", CORE),
    "grad_y_index": ("(p[:, 1:, :] - p[:, :-1, :]) / g.hc[None, :, None]",
                     "(p[:, 1:, :] - p[:, :-1, :]) / g.dy[None, 1:, None]", CORE),
    "nuz_sign": ("nuz = (_zp(fuw) - fuw) / dz", "nuz = (fuw - _zm(fuw)) / dz", CORE),
    "nvx_shift": ("nvx = (_xp(fuv) - fuv) / dx", "nvx = (fuv - _xm(fuv)) / dx", CORE),
    # ADI, tridiagonal solvers, partitioned solve
    "beta_factor": ("beta = RK3_ALPHA[k] * dt * inv_re / 2.0", "beta = RK3_ALPHA[k] * dt * inv_re", CORE),
    "thomas_back_index": ("x[j] = dp[j] - cp[j] * x[j + 1]",
                          "x[j] = dp[j] - cp[j + 1] * x[j + 1]", CORE),
    "cyclic_corner": ("bb[..., n - 1] = b[..., n - 1] - alpha * beta / gam",
                      "bb[..., n - 1] = b[..., n - 1] - alpha * beta * gam", CORE),
    "ppt_perm": ("Zbar = P + E.T @ Ybar", "Zbar = np.eye(len(P)) + E.T @ Ybar", CORE),
    # Poisson and projection
    "dft_sign": ("return np.exp(sign * 2j * math.pi * np.outer(k, k) / n)",
                 "return np.exp(-sign * 2j * math.pi * np.outer(k, k) / n)", CORE),
    "pois_c": ("c[:-1] = 1.0 / (g.dy[:-1] * g.hc)", "c[:-1] = 1.0 / (g.dy[1:] * g.hc)", CORE),
    "wavenumber_period": ("return (2.0 / (h * h)) * (1.0 - np.cos(2.0 * math.pi * l / n))",
                          "return (2.0 / (h * h)) * (1.0 - np.cos(math.pi * l / n))", CORE),
    "project_sign": ("    return u - scale * gx, v - scale * gy, w - scale * gz\n\n\ndef ",
                     "    return u + scale * gx, v - scale * gy, w - scale * gz\n\n\ndef ", CORE),
    "conv_uc_neighbour": ("uc = 0.5 * (u + _xp(u))", "uc = 0.5 * (u + _xm(u))", CORE),
    "conv_w_xface": ("w_xf = 0.5 * (_xm(w) + w)", "w_xf = w", CORE),
    "conv_nvy_spacing": ("nvy[:, 1:-1, :] = (vc[:, 1:, :] ** 2 - vc[:, :-1, :] ** 2) / hc",
                         "nvy[:, 1:-1, :] = (vc[:, 1:, :] ** 2 - vc[:, :-1, :] ** 2) / dy[:, 1:, :]", CORE),
    "div_z_shift": ("+ (_zp(w) - w) / g.dz)", "+ (w - _zm(w)) / g.dz)", CORE),
    "dxx_centre": ("return (_xp(f) - 2.0 * f + _xm(f)) / (g.dx * g.dx)", "return (_xp(f) - 1.0 * f + _xm(f)) / (g.dx * g.dx)", CORE),
    "yrows_A": ("    A = 2.0 / (hm * (hm + hp))\n    C = 2.0 / (hp * (hm + hp))\n    if g.ytop",
                "    A = 2.0 / (hp * (hm + hp))\n    C = 2.0 / (hp * (hm + hp))\n    if g.ytop", CORE),
    "stress_free_top": ("    if g.ytop == 1:\n        C[-1] = 0.0", "    if g.ytop == 1:\n        C[-1] = C[-1]", CORE),
    "rhs_force_coef": ("t = t + alp * fx", "t = t + gam * fx", CORE),
    "rhs_visc_half": ("(alp * inv_re) * L[comp]", "(alp * inv_re / 2.0) * L[comp]", CORE),
    "rhs_pgrad_sign": ("t = -gam * N[comp] - alp * G[comp]", "t = -gam * N[comp] + alp * G[comp]", CORE),
    "pdd_block_offdiag": ("Zb[r:r + 2, r:r + 2] = Z[r:r + 2, r:r + 2]",
                          "Zb[r, r] = Z[r, r]; Zb[r + 1, r + 1] = Z[r + 1, r + 1]", CORE),
    "poisson_scale": ("phi = poisson_solve(g, divergence(g, us, vs, ws) / scale)",
                      "phi = poisson_solve(g, divergence(g, us, vs, ws) * scale)", CORE),
    "pois_a": ("a[1:] = 1.0 / (g.dy[1:] * g.hc)", "a[1:] = 1.0 / (g.dy[:-1] * g.hc)", CORE),
    "adi_x_spacing": ("h = g.dx if direction == 0 else g.dz", "h = g.dz if direction == 0 else g.dz", CORE),
    "nprev_sign": ("t = t - zet * nprev[comp]\n        if comp == 0:\n            t = t + alp * fx\n        t = dt * t\n        if comp == 1:",
                   "t = t + zet * nprev[comp]\n        if comp == 0:\n            t = t + alp * fx\n        t = dt * t\n        if comp == 1:", CORE),
    "p_update_half": ("    if pressure == \"delta\":\n        return p + phi", "    if pressure == \"delta\":\n        return p + 0.5 * phi", CORE + CFL),
    "projection_scale": ("    scale = RK3_ALPHA[k] * dt\n    phi = poisson_solve(g,", "    scale = RK3_GAMMA[k] * dt\n    phi = poisson_solve(g,", CORE + CFL),
    "cyclic_fac_sign": ("fac = (y[..., 0] + beta / gam * y[..., n - 1])", "fac = (y[..., 0] - beta / gam * y[..., n - 1])", CORE),
    "thomas_den": ("den = Bm[j] - A[j] * cp[j - 1]", "den = Bm[j] - Cm[j] * cp[j - 1]", CORE),
    # inflow / convective outflow
    "ghost_coef": ("return np.concatenate([f[:, :, 1:], (2.0 * f_out - f[:, :, -1])[:, :, None]], axis=2)",
                   "return np.concatenate([f[:, :, 1:], (1.0 * f_out)[:, :, None]], axis=2)", BL),
    "adi_3r": ("        b[0] = 1.0 + 3.0 * r\n        b[-1] = 1.0 + 3.0 * r",
               "        b[0] = 1.0 + 2.0 * r\n        b[-1] = 1.0 + 3.0 * r", BL),
    "adi_inc2r": ("d[:, :, -1] += (r if comp == 0 else 2.0 * r) * inc_out", "d[:, :, -1] += r * inc_out", BL),
    "dct_inv": ("    C[:, 1:] *= 2.0\n", "    C[:, 1:] *= 1.0\n", BL),
    "lam_bl": ("lx = (2.0 / (g.dx * g.dx)) * (1.0 - np.cos(math.pi * np.arange(g.nx) / g.nx))",
               "lx = (2.0 / (g.dx * g.dx)) * (1.0 - np.cos(2 * math.pi * np.arange(g.nx) / g.nx))", BL),
    "flux_area": ("return u_out + (q_in - q_out) / area", "return u_out + (q_in - q_out) / (2 * area)", BL),
    "fuv_out": ('fuv_out = uo_yf * bl["v_out"]', 'fuv_out = uo_yf * bl["v_in"]', BL),
    "inflow_ghost": ("return np.concatenate([(2.0 * f_in - f[:, :, 0])[:, :, None], f[:, :, :-1]], axis=2)",
                     "return np.concatenate([(1.0 * f_in)[:, :, None], f[:, :, :-1]], axis=2)", BL),
    "outflow_u_next": ('return np.concatenate([u[:, :, 1:], bl["u_out"][:, :, None]], axis=2)',
                       'return np.concatenate([u[:, :, 1:], u[:, :, -1:]], axis=2)', BL),
    "outflow_v_spacing": ('new["v_out"] = bl["v_out"] - c * (bl["v_out"] - v[:, :, -1]) / (0.5 * g.dx)',
                          'new["v_out"] = bl["v_out"] - c * (bl["v_out"] - v[:, :, -1]) / g.dx', BL),
    "outflow_upwind_sign": ('new["u_out"] = bl["u_out"] - c * (bl["u_out"] - u[:, :, -1]) / g.dx',
                            'new["u_out"] = bl["u_out"] + c * (bl["u_out"] - u[:, :, -1]) / g.dx', BL),
    "inflow_row_identity": ("        a[0], b[0], c[0] = 0.0, 1.0, 0.0\n", "        a[0], b[0], c[0] = 0.0, 1.0, -r\n", BL),
    "bl_v_xface": ('v_xf = 0.5 * (_xprev_c(v, bl["v_in"]) + v)', 'v_xf = 0.5 * (_xm(v) + v)', BL),
    "bl_fuw_out": ('fuw_out = uo_zf * bl["w_out"]', 'fuw_out = uo_zf * bl["w_in"]', BL),
    "bl_grad_inflow": ("    gx[:, :, 0] = 0.0\n    gy = np.zeros((g.nz, g.ny + 1, g.nx))\n    gy[:, 1:-1, :] = (p[:, 1:, :] - p[:, :-1, :]) / g.hc[None, :, None]\n    gz = (p - _zm(p)) / g.dz\n    return gx, gy, gz\n\n\ndef divergence_bl",
                       "    gx[:, :, 0] = gx[:, :, 0]\n    gy = np.zeros((g.nz, g.ny + 1, g.nx))\n    gy[:, 1:-1, :] = (p[:, 1:, :] - p[:, :-1, :]) / g.hc[None, :, None]\n    gz = (p - _zm(p)) / g.dz\n    return gx, gy, gz\n\n\ndef divergence_bl", BL),
    "bl_div_outflow": ("return ((_xnext_u(u, bl) - u) / g.dx", "return ((_xp(u) - u) / g.dx", BL),
    "bl_lap_v_ghost": ('Lv = (_xnext_c(v, bl["v_out"]) - 2.0 * v + _xprev_c(v, bl["v_in"])) / h2',
                       'Lv = (_xp(v) - 2.0 * v + _xprev_c(v, bl["v_in"])) / h2', BL),
    "bl_rhs_inflow_r": ("        if comp == 0:\n            t[:, :, 0] = 0.0\n", "        if comp == 0:\n            t[:, :, 0] = t[:, :, 0]\n", BL),
    "bl_flux_weights": ("w = g.dy[None, :] * g.dz\n", "w = g.dz\n", BL),
    "bl_flux_before_poisson": ('    bl_new["u_out"] = flux_correct_outflow(g, u[:, :, 0], bl_new["u_out"])\n    phi = poisson_solve_bl',
                               '    phi = poisson_solve_bl', BL),
    "bl_ycoeff_gauge": ("    B[0, 0, 0] = 1.0\n    C[0, 0, 0] = 0.0\n    d = d.copy()\n    d[0, 0, 0] = 0.0\n    ph = np.moveaxis(thomas(A, B, C, d), -1, 1)\n    ph = dft(ph, 0, +1) / g.nz",
                        "    B[0, 0, 0] = 1.0\n    C[0, 0, 0] = 0.0\n    d = d.copy()\n    ph = np.moveaxis(thomas(A, B, C, d), -1, 1)\n    ph = dft(ph, 0, +1) / g.nz", BL),
    # fixed-CFL rate and the Kim-Moin update
    "rate_vface": ("vc = 0.5 * (v[:, :-1, :] + v[:, 1:, :])\n    c = np.abs(u) / g.dx",
                   "vc = v[:, :-1, :]\n    c = np.abs(u) / g.dx", CFL),
    "rate_dz": ("np.abs(w) / g.dz\n    return float(c.max())", "np.abs(w) / g.dx\n    return float(c.max())", CFL),
    "rate_noabs": ("c = np.abs(u) / g.dx", "c = u / g.dx", CFL),
    "km_sign": ("return p + phi - beta * lap_phi", "return p + phi + beta * lap_phi", CFL),
    "km_beta2": ("return p + phi - beta * lap_phi", "return p + phi - 2.0 * beta * lap_phi", CFL),
    "cfl_dt_frozen": ('dt = cfl / convective_rate(g, s["u"], s["v"], s["w"])',
                      'dt = cfl / convective_rate(g, state["u"], state["v"], state["w"])', CFL),
    "km_operator": ("lap = divergence(g, *gradient(g, phi)) if pressure != \"delta\" else None",
                    "lap = laplacian(g, phi, phi, phi)[0] if pressure != \"delta\" else None", CFL),
    # recycling inflow
    "lund_b": ("def lund_weight(eta, a=4.0, b=0.2):", "def lund_weight(eta, a=4.0, b=0.3):", RCY),
    "inner_outer_swap": ("    Ui = gamma * sample_c(U[None, :], gamma * yc)\n    Uo = gamma * sample_c(U[None, :], r * yc) + (1.0 - gamma) * u_inf",
                         "    Ui = gamma * sample_c(U[None, :], r * yc)\n    Uo = gamma * sample_c(U[None, :], gamma * yc) + (1.0 - gamma) * u_inf", RCY),
    "outer_defect": ("+ (1.0 - gamma) * u_inf\n    ui =", "+ (gamma - 1.0) * u_inf\n    ui =", RCY),
    "fluct_nogamma": ("    uo = gamma * sample_c(up, r * yc)\n", "    uo = sample_c(up, r * yc)\n", RCY),
    "w_mean_kept": ("    wp = w_r - Wm[None, :]\n", "    wp = w_r + 0.0 * Wm[None, :]\n", RCY),
    "delta99_target": ("target = 0.99 * u_inf", "target = 0.95 * u_inf", RCY),
    "gamma_exp": ("gamma = (delta_rec / delta_inl) ** 0.125", "gamma = (delta_rec / delta_inl) ** 0.1", RCY),
    "recycle_v_avg": ("v_r = 0.5 * (v[:, :, i_r - 1] + v[:, :, i_r])", "v_r = v[:, :, i_r]", RCY),
    "grid_hc": ("self.hc = self.yc[1:] - self.yc[:-1]", "self.hc = self.dy[1:]", CORE),
    "grid_yc": ("self.yc = 0.5 * (self.yf[:-1] + self.yf[1:])", "self.yc = self.yf[:-1]", CORE),
    "dense_cyclic_corner": ("        A[0, n - 1] = a[0]\n        A[n - 1, 0] = c[n - 1]", "        A[0, n - 1] = c[n - 1]\n        A[n - 1, 0] = a[0]", CORE),
    "partition_first_row": ("        first = ((r + 1) % p) * m", "        first = (r + 1) * m - 1 if r + 1 < p else 0", CORE),
    "partition_V_pairing": ("        V[first, 2 * r] = A[first, last]", "        V[first, 2 * r] = A[last, first]", CORE),
    "swap_perm_identity": ("        P[r, r + 1] = 1.0\n        P[r + 1, r] = 1.0", "        P[r, r] = 1.0\n        P[r + 1, r + 1] = 1.0", CORE),
    "adi_drops_z": ("        x = adi_sweep(g, r, 0, comp, beta)\n        x = adi_sweep(g, x, 1, comp, beta)\n        x = adi_sweep(g, x, 2, comp, beta)\n        out.append(x)\n    return out",
                      "        x = adi_sweep(g, r, 0, comp, beta)\n        x = adi_sweep(g, x, 1, comp, beta)\n        out.append(x)\n    return out", CORE),
    "volumes_v": ("hv[1:-1] = self.hc", "hv[1:-1] = self.dy[1:]", CORE),
    "yrows_face_C": ("    hp = g.dy[1:]\n    A = 2.0 / (hm * (hm + hp))\n    C = 2.0 / (hp * (hm + hp))",
                     "    hp = g.dy[1:]\n    A = 2.0 / (hm * (hm + hp))\n    C = 2.0 / (hm * (hm + hp))", CORE),
    "dyy_centre_shift": ("    fp[:, :-1, :] = f[:, 1:, :]", "    fp[:, :-1, :] = f[:, :-1, :]", CORE),
    "dyy_face_shift": ("+ C[None, :, None] * f[:, 2:, :])", "+ C[None, :, None] * f[:, 1:-1, :])", CORE),
    "pdd_drop_block": ("        Zo[r:r + 2, r:r + 2] = 0.0", "        Zo[r, r] = 0.0", CORE),
    "dct2_half_shift": ("return np.cos(math.pi * l * (2 * i + 1) / (2 * n))", "return np.cos(math.pi * l * (2 * i) / (2 * n))", BL),
    "recycle_not_applied": ("        u[:, :, 0] = u_in\n", "        u[:, :, 0] = u[:, :, 0]\n", RCY),
    "periodic_gauge": ("    d[0, 0, 0] = 0.0\n    ph = thomas(A, B, C, d)\n    ph = np.moveaxis(ph, -1, 1)",
                       "    ph = thomas(A, B, C, d)\n    ph = np.moveaxis(ph, -1, 1)", CORE + BL),
    "step_two_substeps": ("    for _ in range(nsteps):\n        for k in range(3):\n            s = substep(g, s, k, dt, re, fx, pressure)",
                          "    for _ in range(nsteps):\n        for k in range(2):\n            s = substep(g, s, k, dt, re, fx, pressure)", CORE),
    "conv_fvw_no_interp": ("    fvw = v_zf * w_yf\n    nvz = (_zp(fvw) - fvw) / dz\n    Nv = nvx + nvy + nvz\n    Nv[:, 0, :] = 0.0\n    Nv[:, -1, :] = 0.0\n    # ---- Nw",
                           "    fvw = v * w_yf\n    nvz = (_zp(fvw) - fvw) / dz\n    Nv = nvx + nvy + nvz\n    Nv[:, 0, :] = 0.0\n    Nv[:, -1, :] = 0.0\n    # ---- Nw", CORE),
    "inverse_dft_norm": ("    phi = dft(dft(ph, 0, +1), 2, +1) / (g.nx * g.nz)", "    phi = dft(dft(ph, 0, +1), 2, +1) / g.nx", CORE),
    "make_div_free_scale": ("    return project(g, u, v, w, phi, 1.0)", "    return project(g, u, v, w, phi, 0.5)", CORE),
    "recycle_v_inner_scale": ("    vi = gamma * _interp_rows(gamma * yf, yf, vp)", "    vi = _interp_rows(gamma * yf, yf, vp)", RCY),
    "recycle_v_outer_height": ("    Vo = _interp_rows(r * yf, yf, V[None, :])", "    Vo = _interp_rows(gamma * yf, yf, V[None, :])", RCY),
    "recycle_blend_swap": ("        return (1.0 - wgt) * inner + wgt * outer", "        return wgt * inner + (1.0 - wgt) * outer", RCY),
    "recycle_blend_eta": ("        wgt = lund_weight(y / delta_inl)[None, :]", "        wgt = lund_weight(y / delta_rec)[None, :]", RCY),
    "recycle_wall_sample": ("        z1 = np.zeros((f2d.shape[0], 1))", "        z1 = f2d[:, :1]", RCY),
    "recycle_w_avg": ("w_r = 0.5 * (w[:, :, i_r - 1] + w[:, :, i_r])", "w_r = w[:, :, i_r]", RCY),
    "delta99_interp": ("return yc[j - 1] + (target - U[j - 1]) * (yc[j] - yc[j - 1]) / (U[j] - U[j - 1])",
                       "return yc[j - 1] + (target - U[j - 1]) * (yc[j] - yc[j - 1]) / U[j]", RCY),
    "lund_weight_top": ("    return np.where(eta > 1.0, 1.0, wgt)", "    return wgt", RCY),
}


def _copy_tree(dst):
    """The oracle, the pin tests and the input generators (pure Python) in dst."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in os.listdir(os.path.join(ROOT, "tests")):
        if f in ("__init__.py", "conftest.py") or (f.startswith("test_oracle_") and f.endswith(".py")):
            shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    os.makedirs(os.path.join(dst, "paper_1812_01178_gb300"))
    for f in ("__init__.py", "inputs.py"):
        shutil.copy(os.path.join(ROOT, "paper_1812_01178_gb300", f), os.path.join(dst, "paper_1812_01178_gb300", f))


def _run(tmp, name):
    a, b, files = MUTANTS[name]
    d = os.path.join(tmp, name)
    _copy_tree(d)
    src = open(ORACLE).read()
    open(os.path.join(d, "oracle", "ns_oracle.py"), "w").write(src.replace(a, b, 1))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-p", "no:cacheprovider", "-x", "-q", "-m", "not gpu"] + files,
                       cwd=d, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, (r.stdout.strip().splitlines() or [""])[-1]


def test_every_mutant_text_is_in_the_oracle():
    src = open(ORACLE).read()
    for name, (a, b, _) in MUTANTS.items():
        assert src.count(a) >= 1 and a != b, name


def test_the_pins_catch_every_mutant(tmp_path):
    names = list(MUTANTS)
    with ThreadPoolExecutor(max_workers=max(2, min(len(names), os.cpu_count() or 2))) as ex:
        results = list(ex.map(lambda n: _run(str(tmp_path), n), names))
    missed = [(n, last) for n, rc, last in results if rc == 0]
    assert not missed, missed
    # exit code 1 = tests failed (not a collection or usage error)
    errors = [(n, rc, last) for n, rc, last in results if rc not in (1,)]
    assert not errors, errors


def test_the_unmutated_copy_passes(tmp_path):
    d = str(tmp_path / "clean")
    _copy_tree(d)
    r = subprocess.run([sys.executable, "-m", "pytest", "-p", "no:cacheprovider", "-x", "-q", "-m", "not gpu"]
                       + CORE + BL + CFL + RCY, cwd=d, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONDONTWRITEBYTECODE="1"))
    assert r.returncode == 0, r.stdout[-2000:]
