"""Mutation check of the oracle's pins (no GPU): a plausible mistake planted anywhere in the
oracle must fail at least one pin.

Each mutant is a copy of oracle/nsk_oracle.c (compiled into a temporary library with the
oracle's own flags), or of one of the oracle's Python modules, with one slip of the kind a hand
translation of the paper makes (a dropped term, a wrong sign, index or factor, a transposed
operand, a one-sided flux where the method takes a mean). A child process points the oracle at
the mutant and runs the pin files of the part it touches; the child must report failing tests
(exit status 1). The unmutated copy, run the same way, must pass every one of those files, so a
failing harness cannot pass for a caught mutant. Nothing is written under oracle/.
"""
import os
import subprocess
import sys
import textwrap
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
SRC = ROOT / "oracle" / "nsk_oracle.c"
HDR = ROOT / "oracle" / "nsk_oracle.h"

CORE = ["tests/test_oracle_pins.py", "tests/test_oracle_mms.py"]
NSK = CORE + ["tests/test_oracle_nsk.py"]
HLLC = ["tests/test_oracle_hllc.py"]
FV = ["tests/test_oracle_fv.py"]

# name: (source text, its replacement, which occurrence, how many occurrences, pin files)
MUTANTS = {
    # thermodynamics and fluxes of relaxation model II (Secs. 2.1, 2.3)
    "vdw_attraction_sign": ("- VDW_A * rho * rho;\n}\n\n/* dp/drho", "+ VDW_A * rho * rho;\n}\n\n/* dp/drho", 0, 1, CORE),
    "modified_pressure_dropped": ("return orc_pressure(s->T, rho) + s->alpha * rho * rho / 2.0;",
                                  "return orc_pressure(s->T, rho);", 0, 1, CORE),
    "momentum_source_dropped": ("R[(1 + a) * nn + p] += s->alpha * rho * Q[(a * nw + d) * nn + p];",
                                "R[(1 + a) * nn + p] += 0.0 * Q[(a * nw + d) * nn + p];", 0, 1, CORE),
    "relaxation_source_sign": ("s->alpha / s->beta * (rho - c);", "s->alpha / s->beta * (c - rho);", 0, 1, CORE),
    "stress_without_transpose": ("double t = Q[k * (d + 1) + a] + Q[a * (d + 1) + k];",
                                 "double t = 2.0 * Q[k * (d + 1) + a];", 0, 2, CORE),
    "stress_divergence_factor": ("if (a == k) t -= 2.0 / 3.0 * div;", "if (a == k) t -= 1.0 / 3.0 * div;", 0, 2, CORE),
    "c_diffusion_without_beta": ("f[d + 1] = s->kappa / s->beta * Q[k * (d + 1) + d];",
                                 "f[d + 1] = s->kappa * Q[k * (d + 1) + d];", 0, 1, CORE),
    "sound_speed_without_alpha": ("return sqrt(orc_dpressure(s->T, rho) + s->alpha * rho);",
                                  "return sqrt(fabs(orc_dpressure(s->T, rho)));", 0, 1, CORE),
    "lax_friedrichs_sign": ("F[v] -= 0.5 * lam * (UR[v] - UL[v]);", "F[v] += 0.5 * lam * (UR[v] - UL[v]);", 0, 1, CORE),
    "lax_friedrichs_min_speed": ("const double lam = lamL > lamR ? lamL : lamR;",
                                 "const double lam = lamL < lamR ? lamL : lamR;", 0, 1, CORE),
    # the DGSEM operator, BR1 and the time integrator (Sec. 3.1)
    "derivative_matrix_transposed": ("D[i * (N + 1) + j] = lagrange_deriv(N, xi, j, xi[i]);",
                                     "D[j * (N + 1) + i] = lagrange_deriv(N, xi, j, xi[i]);", 0, 1, CORE),
    "volume_weight_index": ("vol += m->w[j] * F[j][v] * m->D[j * np + i];",
                            "vol += m->w[i] * F[j][v] * m->D[j * np + i];", 0, 2, CORE),
    "surface_term_sign": ("R[v * nn + eR * npe + node] += (2.0 / m->h[k]) * Fs[v] * m->Lm[i] / m->w[i];",
                          "R[v * nn + eR * npe + node] -= (2.0 / m->h[k]) * Fs[v] * m->Lm[i] / m->w[i];", 0, 2, CORE),
    "neighbour_trace_side": ("UR[v] = trace(m, U + v * nn, eR, k, n0, -1);",
                             "UR[v] = trace(m, U + v * nn, eR, k, n0, +1);", 0, 2, CORE),
    "viscous_flux_one_sided": ("for (int v = 0; v < nv; ++v) Fs[v] -= 0.5 * (fvL[v] + fvR[v]);",
                               "for (int v = 0; v < nv; ++v) Fs[v] -= fvL[v];", 0, 1, CORE),
    "br1_lifting_one_sided": ("wsm[q] = 0.5 * (wm[q] + wnm[q]);", "wsm[q] = wm[q];", 0, 1, CORE),
    "lifting_volume_sign": ("= (2.0 / m->h[k]) * (surf - vol);\n          }", "= (2.0 / m->h[k]) * (surf + vol);\n          }",
                            0, 1, CORE),
    "lagrange_denominator_sign": ("if (m != j) l *= (x - xi[m]) / (xi[j] - xi[m]);",
                                  "if (m != j) l *= (x - xi[m]) / (xi[m] - xi[j]);", 0, 1, CORE),
    "neighbour_direction": ("int cn = (c + dir + m->ne[k]) % m->ne[k];", "int cn = (c - dir + m->ne[k]) % m->ne[k];",
                            0, 1, CORE),
    "lifting_metric_factor": ("Q[(long)(k * nw + q) * nn + e * npe + node] = (2.0 / m->h[k]) * (surf - vol);",
                              "Q[(long)(k * nw + q) * nn + e * npe + node] = (1.0 / m->h[k]) * (surf - vol);", 0, 1, CORE),
    "volume_metric_factor": ("R[v * nn + e * npe + node] += (2.0 / m->h[k]) * vol / m->w[i];",
                             "R[v * nn + e * npe + node] += (1.0 / m->h[k]) * vol / m->w[i];", 0, 2, CORE),
    "lsrk4_register_skipped": ("U[i] = U[i] + B[stage] * K[i];", "U[i] = U[i] + B[stage] * dt * R[i];", 0, 2, CORE),
    "lsrk4_coefficient_typo": ("B[3] = 3134564353537.0 / 4481467310338.0;", "B[3] = 3134564353537.0 / 4481467301338.0;",
                               0, 1, CORE),
    # time-step bounds (Eq. numerics_dfl and R9) and the diagnostics (Eq. pararelax_elliptical_energy_dynamic)
    "source_bound_constant": ("cfl * 4.6 * s->beta / s->alpha", "cfl * 4.8 * s->beta / s->alpha", 0, 1, CORE),
    "convective_bound_order": ("const double twoNp1 = 2.0 * s->N + 1.0;", "const double twoNp1 = s->N + 1.0;", 0, 1, CORE),
    "parabolic_bound_without_c_diffusion": ("double lamv = s->mu > s->kappa / s->beta ? s->mu : s->kappa / s->beta;",
                                            "double lamv = s->mu;", 0, 1, CORE),
    "energy_kinetic_factor": ("se += wq * (m2 / (2.0 * rho)", "se += wq * (m2 / rho", 0, 1, CORE),
    "energy_capillary_dropped": ("s->kappa / 2.0 * g2);", "0.0 * g2);", 0, 1, CORE),
    "energy_relaxation_factor": ("s->alpha / 2.0 * (rho - c) * (rho - c) +", "s->alpha * (rho - c) * (rho - c) +", 0, 1, CORE),
    "mass_without_node_weight": ("sm += wq * rho;", "sm += J * rho;", 0, 1, CORE),
    "bound_order_2n_minus_1": ("const double twoNp1 = 2.0 * s->N + 1.0;", "const double twoNp1 = 2.0 * s->N - 1.0;",
                               0, 1, CORE),
    "bound_offset_2n_plus_2": ("const double twoNp1 = 2.0 * s->N + 1.0;", "const double twoNp1 = 2.0 * s->N + 2.0;",
                               0, 1, CORE),
    "bound_offset_2n_plus_half": ("const double twoNp1 = 2.0 * s->N + 1.0;", "const double twoNp1 = 2.0 * s->N + 0.5;",
                                  0, 1, CORE),
    "parabolic_bound_offset": ("double dt_visc = lamv > 0.0 ? cfl / (twoNp1 * twoNp1 * lamv * inv_h2) : INFINITY;",
                               "double dt_visc = lamv > 0.0 ? cfl / ((twoNp1 + 1.0) * twoNp1 * lamv * inv_h2) : INFINITY;",
                               0, 1, CORE),
    "convective_bound_offset": ("double dt_conv = cfl / (twoNp1 * lam_max);", "double dt_conv = cfl / ((twoNp1 - 0.5) * lam_max);",
                                0, 1, CORE),
    "energy_momentum_index": ("m2 += U[(1 + a) * nn + p] * U[(1 + a) * nn + p];",
                              "m2 += U[(1 - a) * nn + p] * U[(1 + a) * nn + p];", 0, 1, CORE),
    "l2_without_weights": ("sl += wq * (rho - c) * (rho - c);", "sl += (rho - c) * (rho - c);", 0, 1, CORE),
    # the original NSK equations (Sec. 2.2)
    "korteweg_tensor_sign": ("double tk = -s->kappa * Q[a * (d + 1) + d] * Q[k * (d + 1) + d];",
                             "double tk = s->kappa * Q[a * (d + 1) + d] * Q[k * (d + 1) + d];", 0, 1, NSK),
    "korteweg_gradient_square_factor": ("tk += s->kappa * (rho * lap + 0.5 * g2);", "tk += s->kappa * (rho * lap + g2);",
                                        0, 1, NSK),
    "korteweg_gradient_index": ("double tk = -s->kappa * Q[a * (d + 1) + d] * Q[k * (d + 1) + d];",
                                "double tk = -s->kappa * Q[a * (d - 1) + d] * Q[k * (d + 1) + d];", 0, 1, NSK),
    "second_lifting_one_sided": ("const double gsp = 0.5 * (trace(m, g, e, k, n0, +1) + trace(m, g, eR, k, n0, -1));",
                                 "const double gsp = trace(m, g, e, k, n0, +1);", 0, 1, NSK),
    "nsk_stress_without_transpose": ("double t = Q[k * (d + 1) + a] + Q[a * (d + 1) + k];",
                                     "double t = 2.0 * Q[k * (d + 1) + a];", 1, 2, NSK),
    # HLLC (Sec. 3.1)
    "hllc_star_normal_velocity": ("Us[1 + a] = coef * (a == k ? Ss : UK[1 + a] / UK[0]);",
                                  "Us[1 + a] = coef * (UK[1 + a] / UK[0]);", 0, 1, HLLC),
    "hllc_outer_speed": ("SR = fmax(uL + aL, uR + aR);", "SR = fmax(uL + aL, uR - aR);", 0, 1, HLLC),
    "hllc_supersonic_branch": ("for (int v = 0; v < nv; ++v) F[v] = fL[v];", "for (int v = 0; v < nv; ++v) F[v] = fR[v];",
                               0, 1, HLLC),
    "hllc_contact_side": ("const int left = Ss >= 0.0;", "const int left = Ss < 0.0;", 0, 1, HLLC),
    # FV sub-cells, indicator, switching and Dirichlet boundaries (Sec. 3.2)
    "minmod_inverted": ("return a > 0.0 ? fmin(a, b) : fmax(a, b);", "return a > 0.0 ? fmax(a, b) : fmin(a, b);",
                        0, 1, FV),
    "minmod_left_slope_sum": ("(x->P[j][q] - x->P[j - 1][q]) / dx", "(x->P[j][q] + x->P[j - 1][q]) / dx", 0, 1, FV),
    "boundary_half_width": ("dn[sd] = 0.5 * dx;\n        continue;", "dn[sd] = dx;\n        continue;", 0, 1, FV),
    "subcell_source_one_sided": ("R[nn + p] += s->alpha * U[p] * 0.5 * (gc[j] + gc[j + 1]);",
                                 "R[nn + p] += s->alpha * U[p] * gc[j + 1];", 0, 1, FV),
    "reconstruction_mirrored": ("PL[q] = x->P[j][q] + 0.5 * dx * x->sl[j][q];",
                                "PL[q] = x->P[j][q] - 0.5 * dx * x->sl[j][q];", 0, 1, FV),
    "subcell_viscous_sign": ("for (int v = 0; v < 3; ++v) Fs[j + 1][v] -= fvv[v];",
                             "for (int v = 0; v < 3; ++v) Fs[j + 1][v] += fvv[v];", 0, 1, FV),
    "back_switch_threshold": ("fv[e] && x < f->ind_lower", "fv[e] && x < f->ind_upper", 0, 1, FV),
    "periodic_flux_shifted": ("memcpy(Fh[E], Fh[0], sizeof(double[3]));", "memcpy(Fh[E], Fh[1], sizeof(double[3]));",
                              0, 1, FV),
    "mixed_lifting_without_neighbour": ("ws[sd][1] = 0.5 * (Ui[2] + Uo[2]);", "ws[sd][1] = Ui[2];", 0, 1, FV),
    "indicator_normalisation": ("return log10(uh[N] * uh[N] / tot);",
                                "return log10(uh[N] * uh[N] / (tot - uh[0] * uh[0] + 1e-300));", 0, 1, FV),
    "legendre_modes_not_normalised": ("return sqrt((2.0 * m + 1.0) / 2.0) * P;", "return P;", 0, 1, FV),
    "subcell_mean_factor": ("M[j * np + i] = 0.5 * s;", "M[j * np + i] = s;", 0, 1, FV),
    "subcell_offset": ("const double a = -1.0 + 2.0 * j / np;", "const double a = -1.0 + 2.0 * j / (np + 1);", 0, 1, FV),
    "conversion_matrices_swapped": ("const double* T = to_fv ? M : Minv;", "const double* T = to_fv ? Minv : M;", 0, 1, FV),
    "dirichlet_ghost_gradient_side": ("const double* gL = eL >= 0 ? el[eL].gf[1] : el[eR].gf[0];",
                                      "const double* gL = eL >= 0 ? el[eL].gf[1] : el[eR].gf[1];", 0, 1, FV),
    "dg_neighbour_trace_side": ("fv_dg_trace(&m, U, en, sd ? 0 : 1, Ut);", "fv_dg_trace(&m, U, en, sd ? 1 : 0, Ut);",
                                0, 1, FV),
    "indicator_inverse_mean_transposed": ("rho[i] += Minv[i * np + j] * U[e * np + j];",
                                          "rho[i] += Minv[j * np + i] * U[e * np + j];", 0, 1, FV),
}

ESDIRK = ["tests/test_oracle_esdirk.py"]
CLOSURE = ["tests/test_oracle_closure.py"]

# the oracle's Python modules: name: (module, source text, replacement, occurrence, count, pin files)
PY_MUTANTS = {
    "esdirk_tableau_entry": ("esdirk", "Fr(-1743, 31250)", "Fr(-1743, 31520)", 0, 1, ESDIRK),
    "esdirk_gamma": ("esdirk", "GAMMA = Fr(1, 4)", "GAMMA = Fr(1, 3)", 0, 1, ESDIRK),
    "esdirk_stage_sum_short": ("esdirk", "for j in range(i))", "for j in range(i - 1))", 0, 1, ESDIRK),
    "esdirk_stage_derivative_scale": ("esdirk", "R.append((X - S) / (dt * g))", "R.append((X - S) / dt)", 0, 1, ESDIRK),
    "gmres_givens_sign": ("esdirk", "H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]",
                          "H[j + 1, k] = sn[j] * H[j, k] + cs[j] * H[j + 1, k]", 0, 1, ESDIRK),
    "gmres_stale_residual_estimate": ("esdirk", "if abs(g[k + 1]) <= tol * bn or its >= maxit:\n                break",
                                      "if abs(g[k - 1]) <= tol * bn or its >= maxit:\n                break", 0, 1, ESDIRK),
    "newton_count_lost": ("esdirk", 'st["newton"] += 1', 'st["newton"] += 0', 0, 1, ESDIRK),
    "colouring_too_few": ("esdirk", "for K in range(3, ne + 1):", "for K in range(2, ne + 1):", 0, 1, ESDIRK),
    "preconditioner_sign": ("esdirk", "np.linalg.inv(np.eye(n)[None] - dtg * J)",
                            "np.linalg.inv(np.eye(n)[None] + dtg * J)", 0, 1, ESDIRK),
    "gelu_scale": ("mlp", "return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))", "return 0.5 * z * (1.0 + _erf(z / 2.0))",
                   0, 1, CLOSURE),
    "gelu_grad_term_dropped": ("mlp", " + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)", "", 0, 1, CLOSURE),
    "second_activation_dropped": ("mlp", "h2 = gelu(z2)", "h2 = z2", 0, 1, CLOSURE),
    "loss_mean_over_rows": ("mlp", "n = y.size", "n = y.shape[0]", 0, 1, CLOSURE),
    "backprop_wrong_preactivation": ("mlp", "dz1 = (dz2 @ p[\"W2\"]) * gelu_grad(z1)",
                                     "dz1 = (dz2 @ p[\"W2\"]) * gelu_grad(z2[:, :z1.shape[1]])", 0, 1, CLOSURE),
}

DRIVER = textwrap.dedent('''
    import importlib.util
    import sys
    from pathlib import Path
    root, so, module, path = sys.argv[1], Path(sys.argv[2]), sys.argv[3], sys.argv[4]
    sys.path.insert(0, root)
    import oracle
    oracle.build_oracle = lambda force=False, parallel=False: so
    if module != "-":  # a mutated copy of oracle/<module>.py in place of the module
        spec = importlib.util.spec_from_file_location("oracle." + module, path)
        mod = importlib.util.module_from_spec(spec)
        sys.modules["oracle." + module] = mod
        spec.loader.exec_module(mod)
        setattr(oracle, module, mod)
    import pytest
    sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"] + [root + "/" + f for f in sys.argv[5:]]))
''')


def _mutate(src, old, new, nth):
    i = -1
    for _ in range(nth + 1):
        i = src.index(old, i + 1)
    return src[:i] + new + src[i + len(old):]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = tmp_path_factory.mktemp("mutants")
    (tmp / "drive.py").write_text(DRIVER)
    (tmp / "nsk_oracle.h").write_text(HDR.read_text())
    src = SRC.read_text()

    def compile_c(name, text):
        c = tmp / f"{name}.c"
        c.write_text(text)
        so = tmp / f"lib{name}.so"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(c), "-o", str(so), "-lm"],
                       check=True)
        return so

    control_so = compile_c("control", src)
    # name: (C source text or None for the control library, Python module or "-", its mutated text, pin files)
    jobs = {"control": (None, "-", "", sorted(set(CORE + NSK + HLLC + FV + ESDIRK + CLOSURE)))}
    for name, (old, new, nth, count, files) in MUTANTS.items():
        assert src.count(old) == count, f"{name}: the oracle source changed; update the mutant"
        jobs[name] = (_mutate(src, old, new, nth), "-", "", files)
    for name, (module, old, new, nth, count, files) in PY_MUTANTS.items():
        text = (ROOT / "oracle" / f"{module}.py").read_text()
        assert text.count(old) == count, f"{name}: oracle/{module}.py changed; update the mutant"
        jobs[name] = (None, module, _mutate(text, old, new, nth), files)

    def run(item):
        name, (c_text, module, py_text, files) = item
        so = control_so if c_text is None else compile_c(name, c_text)
        py = tmp / f"{name}_{module}.py"
        if module != "-":
            py.write_text(py_text)
        r = subprocess.run([sys.executable, str(tmp / "drive.py"), str(ROOT), str(so), module, str(py)] + files,
                           cwd=str(tmp), capture_output=True, text=True, timeout=600)
        failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
        return name, (r.returncode, failed[:1], r.stdout[-2000:])

    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(run, jobs.items()))


def test_unmutated_copy_passes_every_pin(outcomes):
    rc, _, out = outcomes["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS) + sorted(PY_MUTANTS))
def test_mutant_fails_a_pin(outcomes, name):
    rc, failed, out = outcomes[name]
    assert rc == 1 and failed, f"{name} survived the pins (exit {rc}):\n{out}"
