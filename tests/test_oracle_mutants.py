"""Plausible mistakes planted in a CPU copy of the oracle must each fail at least one pin.

This shows the pins constrain every part of the oracle: a dropped term, a wrong sign,
index or prefactor, a transposed operand.  Mutants are compiled into a temporary
directory; the oracle source itself is never modified.
"""
import os
import subprocess

import pytest

import oracle_pins as P
from oracle import build as obuild
from oracle.oracle import Oracle

MUTANTS = {
    "nonlinear_sign": ("double f = c * c * c - c;", "double f = c - c * c * c;"),
    "gamma_sign": ("mu[p] = f - gamma * or_lap_at", "mu[p] = f + gamma * or_lap_at"),
    "lap_y_uses_hx": ("- 2.0 * c) / (hy * hy);", "- 2.0 * c) / (hx * hx);"),
    "lap_drop_center": ("+ v[(size_t)jm * nx + i] - 2.0 * c)", "+ v[(size_t)jm * nx + i] - 1.0 * c)"),
    "rhs_no_dt": ("R[(size_t)j * nx + i] = dt * or_lap_at", "R[(size_t)j * nx + i] = or_lap_at"),
    "sx_wrong_power": ("double sx = gamma * dt / (hx * hx * hx * hx);", "double sx = gamma * dt / (hx * hx * hx);"),
    "sy_uses_hx": ("double sy = gamma * dt / (hy * hy * hy * hy);", "double sy = gamma * dt / (hx * hx * hx * hx);"),
    "penta_offdiag": ("return -4.0 * s;", "return -3.0 * s;"),
    "penta_diag": ("return 1.0 + 6.0 * s;", "return 1.0 + 4.0 * s;"),
    "schur_sign": ("acc -= or_penta_coef(n, s, m + a, j) * rhs[(size_t)j * 3 + b];",
                   "acc += or_penta_coef(n, s, m + a, j) * rhs[(size_t)j * 3 + b];"),
    "backsub_drop_border": ("- rhs[(size_t)i * 3 + 1] * xm1;", ";"),
    "elim_pivot_row": ("double l = band[(size_t)i * 5 + 2 + (k - i)] / piv;",
                       "double l = band[(size_t)i * 5 + 2 + (k - i)] / (piv + 1e-3);"),
    "update_sign": ("C[(size_t)j * nx + i] + lout[j]", "C[(size_t)j * nx + i] - lout[j]"),
    "rows_cols_swapped_s": ("rc = or_cyclic_penta_solve(nx, sx, lin, lout);", "rc = or_cyclic_penta_solve(nx, sy, lin, lout);"),
    "bulk_half": ("sF += 0.25 * w * w", "sF += 0.5 * w * w"),
    "grad_no_half": ("+ 0.5 * gamma * (cx * cx + cy * cy)", "+ gamma * (cx * cx + cy * cy)"),
    "grad_drop_y": ("(cx * cx + cy * cy)", "(cx * cx)"),
    "dFdt_sign": ("*dFdt = -(hx * hy * sD);", "*dFdt = (hx * hy * sD);"),
    "dFdt_uses_C": ("double mx = (mu[(size_t)j * nx + ip] - mu[p]) / hx;",
                    "double mx = (C[(size_t)j * nx + ip] - C[p]) / hx;"),
    "beta_sign": ("return -(t / F) * dFdt;", "return (t / F) * dFdt;"),
    "time_offset": ("double t = (double)n * dt;", "double t = (double)(n + 1) * dt;"),
    "window_strict": ("if (t >= t1) {", "if (t > t1) {"),
    "noise_amplitude": ("0.1 * (2.0 * u - 1.0)", "0.1 * (u - 0.5)"),
    "counter_transposed": ("(uint64_t)j * (uint64_t)nx + (uint64_t)i", "(uint64_t)i * (uint64_t)ny + (uint64_t)j"),
    "mix_constant": ("0xbf58476d1ce4e5b9ULL", "0xbf58476d1ce4e5b8ULL"),
    "uniform_bits": ("or_splitmix64(seed, k) >> 11", "or_splitmix64(seed, k) >> 12"),
    "sample_after_update": ("int take = (n % every) == 0;", "int take = ((n + 1) % every) == 0;"),
    "moment_raw": ("double d = b - mu1;", "double d = b;"),
    "moment_unbiased": ("c2 / (double)count : NAN;", "c2 / (double)(count - 1) : NAN;"),
    "mu3_sign": ("c3 += d * d * d;", "c3 -= d * d * d;"),
    "mu4_power": ("c4 += d * d * d * d;", "c4 += d * d * d;"),
    "moment_counts_inf": ("if (isfinite(b)) {\n        sum += b;", "if (!isnan(b)) {\n        sum += b;"),
    "hist_counts_inf": ("if (!isfinite(b)) continue;", "if (isnan(b)) continue;"),
    "hist_lower_edge": ("if (b < lo) {", "if (b <= lo) {"),
    "hist_round": ("double k = floor((b - lo) / w);", "double k = round((b - lo) / w);"),
    "trend_rectangle": ("integral += 0.5 * (t[s + 1] - t[s]) * (mu1[s] + mu1[s + 1]);",
                        "integral += (t[s + 1] - t[s]) * mu1[s];"),
    "trend_span": ("integral / (tb - ta)", "integral / (t2 - t1)"),
    "fit_drops_t": ("stm += t[s] * mu2[s];", "stm += mu2[s];"),
    "fit_window_strict": ("if (t[s] >= tf1 && t[s] <= tf2) {", "if (t[s] > tf1 && t[s] <= tf2) {"),
    "restrict_offset": ("fine[(size_t)(2 * j) * nx + 2 * i + 1] +", "fine[(size_t)(2 * j) * nx + 2 * i + 2] +"),
    "restrict_no_abs": ("sum += fabs(r - coarse[(size_t)j * mx + i]);", "sum += r - coarse[(size_t)j * mx + i];"),
    "restrict_half": ("double r = 0.25 * (fine[", "double r = 0.5 * (fine["),
    "restrict_norm_fine": ("return sum / ((double)mx * (double)my);", "return sum / ((double)nx * (double)my);"),
    "restrict_transposed": ("sum += fabs(r - coarse[(size_t)j * mx + i]);", "sum += fabs(r - coarse[(size_t)i * my + j]);"),
    "drop_rhs_sign": ("(-1.0 / (R[i] * R[i]) + u / R[i])", "(1.0 / (R[i] * R[i]) + u / R[i])"),
    "drop_u_counts_twice": ("alive += 1.0;", "alive += 2.0;"),
    "drop_heaviside_shift": ("(R[i] + eps > 0.0) ?", "(R[i] - eps > 0.0) ?"),
    "drop_F_no_half": ("f += 0.5 * R[i] * R[i];", "f += R[i] * R[i];"),
    "drop_dFdt_sign": ("*dFdt = -d;", "*dFdt = d;"),
    "drop_dFdt_u_sign": ("double g = 1.0 - u * R[i];", "double g = 1.0 + u * R[i];"),
    "dp_a53": ("64448.0 / 6561.0", "64448.0 / 6562.0"),
    "dp_a32": ("{3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0}", "{3.0 / 40.0, 9.0 / 41.0, 0, 0, 0, 0}"),
    "dp_b3": ("500.0 / 1113.0", "500.0 / 1112.0"),
    "dp_bs3": ("7571.0 / 16695.0", "7571.0 / 16696.0"),
    "dp_c5": ("8.0 / 9.0, 1.0, 1.0}", "7.0 / 9.0, 1.0, 1.0}"),
    "dp_no_fsal": ("memcpy(k, k + (size_t)6 * n, sizeof(double) * (size_t)n);", ";"),
    "dp_stage_h": ("ys[i] = y[i] + h * acc;", "ys[i] = y[i] + 0.5 * h * acc;"),
}


@pytest.fixture(scope="module")
def source():
    with open(obuild.SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, "mutation anchor must occur exactly once: %r" % old
    src = tmp_path / "mut.c"
    src.write_text(source.replace(old, new))
    lib = tmp_path / ("libmut_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-o", str(lib),
                    str(src), "-lm"], check=True)
    orc = Oracle(str(lib))
    failed = []
    for pin in P.ALL_PINS:
        try:
            pin(orc)
        except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
            failed.append(pin.__name__)
    assert failed, "mutant %s passed every pin" % name
