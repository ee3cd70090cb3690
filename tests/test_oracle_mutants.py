"""The oracle's pins have teeth: planted mistakes are caught (no GPU).

Each case copies the C oracle, plants one plausible mistake in it (a sign,
a factor, a dropped term, a wrong index, a swapped argument), builds the
mutant with gcc, and runs in a fresh process the pins of
``test_oracle_pins.py`` that should catch it, with the oracle wrapper
pointed at the mutant (several mutants at a time).  The pins must fail (pytest exit status 1: failures,
not errors).  A control run of the same pins against the unchanged source
must pass, so that the failures come from the mistakes and not from the
harness.  The PyTorch statement of the discrete adjoint (oracle/adjoint.py)
gets the same treatment against its own pins.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(REPO, "tests")
SRC = os.path.join(REPO, "oracle", "lbm_oracle.c")
PINS = os.path.join(TESTS, "test_oracle_pins.py")

# (name, text in the oracle, planted replacement, pins expected to catch it)
MUTANTS = [
    ("relaxation_rate", "(1.0 - 1.0 / tau) * L->w[i] * QP", "(1.0 - 0.5 / tau) * L->w[i] * QP",
     "test_shear_wave_decay_gives_lattice_viscosity"),
    ("force_term_half", "+ 0.5 * force_term(L, i, u, F);", "+ 1.0 * force_term(L, i, u, F);",
     "test_collision_moments_match_bgk_with_force"),
    ("shan_chen_sign", "T[T_SC][a][d] = -p->G * r[a] * ga;", "T[T_SC][a][d] = p->G * r[a] * ga;",
     "test_shan_chen_force_on_cosine_field"),
    ("csf_curvature_sign", "p->kappa * (-div)", "p->kappa * (div)",
     "test_csf_force_on_cylinder_matches_continuum"),
    ("anisotropy_minus_one", "double am1 = cv->aniso - 1.0;", "double am1 = cv->aniso;",
     "test_tensorial_resistivity_direction"),
    ("kozeny_carman_power", "(180.0 * (1.0 - phi) * (1.0 - phi))", "(180.0 * (1.0 - phi))",
     "test_darcy_uniform_gray"),
    ("hysteresis_threshold", "if (st->wetflag[c] && s < p->s_lo) {", "if (st->wetflag[c] && s < p->s_hi) {",
     "test_residual_hysteresis_switches"),
    ("bounce_back_slot", "st->f[((long)a * Q + opp[i]) * n + c]", "st->f[((long)a * Q + i) * n + c]",
     "test_poiseuille_profile"),
    ("porosity_gradient_scale", "L->w[i] * (vp - vm) * L->cv[i][d] / CS2;", "L->w[i] * (vp - vm) * L->cv[i][d];",
     "test_principal_axis_on_cosine_porosity"),
    ("d2q9_diagonal_weight", "(len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0)", "(len2 == 1 ? 1.0 / 9.0 : 1.0 / 18.0)",
     "test_d2q9_is_the_plane_projection_of_d3q19_at_unit_tau"),
    ("reservoirs_swapped", "return st->type[c] == INLET ? st->p.rho_in[a] : st->p.rho_out[a];",
     "return st->type[c] == INLET ? st->p.rho_out[a] : st->p.rho_in[a];",
     "test_darcy_between_pressure_reservoirs"),
    ("leverett_square_root", "return sqrt((kref / cv->phi_ref) / (k / phi));",
     "return (kref / cv->phi_ref) / (k / phi);", "test_leverett_invariance_and_residual_crossings"),
    ("thomeer_log_base", "double e = -cv->thomeer_g / log(1.0 - se);",
     "double e = -cv->thomeer_g / log10(1.0 - se);", "test_thomeer_capillary_pressure_inside_the_curve"),
    ("thomeer_crossing_sign", "1.0 - exp(-cv->thomeer_g / log10(ratio))", "1.0 - exp(cv->thomeer_g / log10(ratio))",
     "test_thomeer_residual_crossings"),
    ("mss_direction", "double sgn = a == w ? 1.0 : -1.0;", "double sgn = a == w ? -1.0 : 1.0;",
     "test_mass_sink_source_special_cases"),
    ("mss_background", "double I = (4.0 * rw * rn - Ib) / (1.0 - Ib);", "double I = (4.0 * rw * rn) / (1.0 - Ib);",
     "test_mass_sink_source_special_cases"),
    ("saturation_weight", "double phc = type[c] == GRAY ? phi[c] : 1.0;", "double phc = 1.0;",
     "test_observables_are_plain_sums"),
    ("capillary_sign", "T[T_CAP][a][d] = -Pc * (r[a] / rt)", "T[T_CAP][a][d] = Pc * (r[a] / rt)",
     "test_capillary_force_flat_interface_telescopes"),
    ("drag_implicit_half", "A[a][b] = (a == b ? rt : 0.0) + 0.5 * R[a][b];",
     "A[a][b] = (a == b ? rt : 0.0) + 1.0 * R[a][b];", "test_darcy_uniform_gray"),
    ("corey_exponents_swapped", "kr[w] = pow(se, cv->nw);", "kr[w] = pow(se, cv->nn);",
     "test_two_component_darcy_with_corey_permeabilities"),
    ("wall_density_of_other_component", "return is_wall(st, m) ? st->p.rho_wall[a] : st->rho[a][m];",
     "return is_wall(st, m) ? st->p.rho_wall[1 - a] : st->rho[a][m];", "test_shan_chen_force_next_to_a_wall"),
    ("velocity_half_force", "uc[d] = (jc[d] + 0.5 * Ft) / rt;", "uc[d] = (jc[d] + 1.0 * Ft) / rt;",
     "test_poiseuille_profile"),
    ("csf_phi_avg", "(st->grad[a][d * n + c] / p->phi_avg[a])", "(st->grad[a][d * n + c] * p->phi_avg[a])",
     "test_csf_force_on_cylinder_matches_continuum"),
    ("atwood_cut_inverted", "(fabs(At_c) <= p->at_cut)", "(fabs(At_c) >= p->at_cut)",
     "test_capillary_force_flat_interface_telescopes"),
    ("hermite_trace_dropped", "(L->cv[i][a] * L->cv[i][b] - (a == b ? CS2 : 0.0)) * P[a][b]",
     "(L->cv[i][a] * L->cv[i][b]) * P[a][b]", "test_collision_moments_match_bgk_with_force"),
    ("csf_region_inverted", "(p->csf_everywhere || gray)", "(p->csf_everywhere || !gray)",
     "test_csf_acts_in_gray_cells_only_unless_everywhere"),
    ("residual_crossings_swapped", "sw_at_pressure(cv, lamL, cv->f_max * pc_pm);",
     "sw_at_pressure(cv, lamL, cv->f_min * pc_pm);", "test_leverett_invariance_and_residual_crossings"),
    ("leverett_reference_porosity", "double kref = kozeny_carman(cv, cv->phi_ref);",
     "double kref = kozeny_carman(cv, phi);", "test_leverett_invariance_and_residual_crossings"),
    ("outlet_plane", "if (x == nx - 1) fout += u0;", "if (x == 0) fout += u0;",
     "test_observables_are_plain_sums"),
    ("gradient_weight_dropped", "M[a][b] = acc + st->p.c_g * g[a] * g[b];", "M[a][b] = acc + g[a] * g[b];",
     "test_principal_axis_on_cosine_porosity"),
    ("hessian_cross_factor", "H[a][b] = H[b][a] = 0.25 * (pp - pm - mp + mm);",
     "H[a][b] = H[b][a] = 0.5 * (pp - pm - mp + mm);", "test_principal_axis_on_cosine_porosity"),
    ("kozeny_d_squared", "return cv->kc_d * cv->kc_d * phi * phi * phi", "return cv->kc_d * phi * phi * phi",
     "test_two_component_darcy_with_corey_permeabilities"),
    ("probe_inside_outside", "if (r2 < probe[3] * probe[3]) { pin += pr; nin += 1; }",
     "if (r2 > probe[3] * probe[3]) { pin += pr; nin += 1; }", "test_observables_are_plain_sums"),
    ("mss_not_rest_equilibrium", "st->f[((long)a * Q + i) * n + c] = fout[i] + sgn * L->w[i] * dm;",
     "st->f[((long)a * Q + i) * n + c] = fout[i] + sgn * dm / Q;", "test_mass_sink_source_special_cases"),
    ("curvature_normal_term_sign", "div = (H[0][0] + H[1][1] + H[2][2]) / s - gHg / (s * s * s);",
     "div = (H[0][0] + H[1][1] + H[2][2]) / s + gHg / (s * s * s);",
     "test_csf_force_on_cylinder_matches_continuum"),
    ("hessian_trace_part", "(L->cv[i][d] * L->cv[i][e] - (d == e && d < L->dim ? CS2 : 0.0)) * df",
     "(L->cv[i][d] * L->cv[i][e]) * df", "test_csf_force_on_cylinder_matches_continuum"),
    ("hessian_identity_of_3d_in_2d", "(d == e && d < L->dim ? CS2 : 0.0)", "(d == e && d < 3 ? CS2 : 0.0)",
     "test_csf_force_on_cylinder_matches_continuum"),
]


def _build(tmp_path, text):
    c = tmp_path / "oracle_variant.c"
    c.write_text(text)
    so = tmp_path / "liborc_variant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(c), "-o", str(so), "-lm"],
                   check=True, capture_output=True)
    return str(so)


def _run_pins(so, pins):
    code = (f"import sys; sys.path[:0] = [{REPO!r}, {TESTS!r}]\n"
            f"import oracle\n"
            f"oracle.build = lambda force=False: {so!r}\n"
            f"import pytest\n"
            f"sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', {PINS!r}, '-k', {pins!r}]))\n")
    env = dict(os.environ, OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900, cwd=REPO,
                          env=env)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Builds and runs the control and every mutant, several at a time (each
    is a separate gcc and Python process); returns name -> completed process."""
    with open(SRC) as f:
        text = f.read()
    jobs = [("control", text, " or ".join(m[3] for m in MUTANTS))]
    for name, old, new, pins in MUTANTS:
        assert text.count(old) == 1, f"{name}: the mutated text must occur exactly once"
        jobs.append((name, text.replace(old, new), pins))
    # the directories first, in this thread (tmp_path_factory is not thread-safe)
    dirs = {name: tmp_path_factory.mktemp(name) for name, _, _ in jobs}

    def run(job):
        name, variant, pins = job
        return name, _run_pins(_build(dirs[name], variant), pins)

    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return dict(ex.map(run, jobs))


def test_control_unchanged_oracle_passes_the_pins(outcomes):
    r = outcomes["control"]
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name,pins", [(m[0], m[3]) for m in MUTANTS], ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(outcomes, name, pins):
    r = outcomes[name]
    assert r.returncode == 1, f"{name}: pins {pins} did not fail (exit {r.returncode})\n{r.stdout[-3000:]}"


# ---- the discrete adjoint's PyTorch statement (oracle/adjoint.py) ----------
ADJ_SRC = os.path.join(REPO, "oracle", "adjoint.py")
ADJ_PINS = os.path.join(TESTS, "test_oracle_adjoint.py")
ADJ_MUTANTS = [
    ("eigen_gap_sign", "gap = w[..., 2] - w[..., k]", "gap = w[..., k] - w[..., 2]"),
    ("eigen_direction_dropped", "for k in (0, 1):", "for k in (0,):"),
    ("adjoint_kozeny_power", "return d * d * phi ** 3 / (180.0 * (1.0 - phi) ** 2)",
     "return d * d * phi ** 3 / (180.0 * (1.0 - phi))"),
]


def _run_adjoint_pins(path):
    code = (f"import sys; sys.path[:0] = [{REPO!r}, {TESTS!r}]\n"
            "import importlib.util, oracle\n"
            f"spec = importlib.util.spec_from_file_location('oracle.adjoint', {path!r})\n"
            "mod = importlib.util.module_from_spec(spec); sys.modules['oracle.adjoint'] = mod\n"
            "spec.loader.exec_module(mod); oracle.adjoint = mod\n"
            "import pytest\n"
            f"sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', {ADJ_PINS!r}]))\n")
    env = dict(os.environ, OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900, cwd=REPO,
                          env=env)


@pytest.fixture(scope="module")
def adjoint_outcomes(tmp_path_factory):
    with open(ADJ_SRC) as f:
        text = f.read()
    jobs = [("control", text)]
    for name, old, new in ADJ_MUTANTS:
        assert text.count(old) == 1, f"{name}: the mutated text must occur exactly once"
        jobs.append((name, text.replace(old, new)))
    paths = {}
    for name, variant in jobs:  # files first, in this thread
        path = tmp_path_factory.mktemp("adj_" + name) / "adjoint.py"
        path.write_text(variant)
        paths[name] = str(path)
    with ThreadPoolExecutor(max_workers=max(1, min(4, (os.cpu_count() or 2) // 2))) as ex:
        return dict(zip([j[0] for j in jobs], ex.map(_run_adjoint_pins, [paths[j[0]] for j in jobs])))


def test_control_unchanged_adjoint_statement_passes_its_pins(adjoint_outcomes):
    r = adjoint_outcomes["control"]
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", [m[0] for m in ADJ_MUTANTS])
def test_adjoint_pins_catch_a_planted_mistake(adjoint_outcomes, name):
    r = adjoint_outcomes[name]
    assert r.returncode == 1, f"{name}: the adjoint pins did not fail (exit {r.returncode})\n{r.stdout[-3000:]}"
