"""Planted mistakes in the oracle make its pins fail.

Each case copies the oracle's sources, plants one plausible mistake (a
dropped factor, a flipped sign, a transposed index, a wrong weight), builds
the copy and runs the pins named beside it against the mutant: at least one
must fail.  This shows that the pins constrain the oracle where it could
plausibly go wrong, so that agreement between the CUDA path and the oracle
means agreement with the formulation of arXiv:2505.00384 (Sec. 2 and Sec. 3).
The real oracle is never modified; the mutants live in a temporary folder.
"""
import ctypes
import os
import shutil
import subprocess
import types

import pytest

import oracle as O
import oracle.learned as NL
import test_oracle_imex as I
import test_oracle_learned as TL
import test_oracle_nonconf as NC
import test_oracle_pins as P

ORACLE = os.path.dirname(os.path.abspath(O.__file__))

FLAT = dict(terrain=0)

# (name, file, original text, planted text, [(pin, args)])
C_MUTANTS = [
    ("Gauss weight doubled", "orc.c",
     "w[i] = 1.0 / ((1.0 - t * t) * dP * dP);", "w[i] = 2.0 / ((1.0 - t * t) * dP * dP);",
     [(P.test_gauss_exactness, (3,))]),
    ("central average of p without the 1/2", "orc.c",
     "ph = 0.5 * (pm + dotn(", "ph = (pm + dotn(",
     [(P.test_interior_face_fluxes_closed_form, (1,))]),
    ("transmissive pressure at far-field faces", "orc.c",
     "if (ff) ph = 0.0;", "if (ff) ph = pm;",
     [(P.test_far_field_pressure_flux_closed_form, (1,))]),
    ("far-field faces closed in C", "orc.c",
     "if (nb < 0 && bk == 0) continue;", "if (nb < 0) continue;",
     [(P.test_far_field_divergence_of_constant_field, ())]),
    ("volume term of B with the wrong sign", "orc.c",
     "out[d * n3 + i] -= pq * gd;", "out[d * n3 + i] += pq * gd;",
     [(P.test_single_cell_matrices_closed_form, (1,))]),
    ("transposed inverse Jacobian in B", "orc.c",
     "double gd = g0 * Ji[d] + g1 * Ji[3 + d] + g2 * Ji[6 + d];",
     "double gd = g0 * Ji[3 * d] + g1 * Ji[3 * d + 1] + g2 * Ji[3 * d + 2];",
     [(P.test_B_reproduces_gradient_of_linear_fields, (P.CURVED[0], 1))]),
    ("kappa without the factor gamma", "orc.c",
     "double kf = gamma / (gamma - 1.0);", "double kf = 1.0 / (gamma - 1.0);",
     [(P.test_C_is_minus_kappa_B_transpose_on_curved_walls, (P.CURVED[0],))]),
    ("one-sided kappa in the C face flux", "orc.c",
     "flux = 0.5 * (km * vm + kp * vp);", "flux = 0.5 * (km * vm + km * vp);",
     [(P.test_S_invariants, (FLAT,))]),
    ("alpha instead of alpha^2 in the Helmholtz diagonal", "orc.c",
     "v += alpha * alpha * hq * g2;", "v += alpha * hq * g2;",
     [(P.test_single_cell_matrices_closed_form, (1,))]),
    ("D scaled by 1/gamma in S", "orc.c",
     "cell_M(&S.T, &G, c, 1.0 / (gamma - 1.0), p, loc);", "cell_M(&S.T, &G, c, 1.0 / gamma, p, loc);",
     [(P.test_S_invariants, (FLAT,))]),
    ("Givens rotation with the wrong sign", "orc.c",
     "H[(i + 1) * mm + j] = -sn[i] * a + cs[i] * bb;", "H[(i + 1) * mm + j] = sn[i] * a + cs[i] * bb;",
     [(P.test_fgmres_cycle_minimises_residual_over_krylov_space, (O.PC_NONE, 8))]),
    ("fast-inverse rule weight missing a factor", "orc_core.h",
     "T->wa[p] = T->gaw[i] * T->gaw[j] * T->gaw[k];", "T->wa[p] = T->gaw[i] * T->gaw[j];",
     [(P.test_fast_inverse_is_tensor_product_form, ())]),
    ("face normal along +xi on both sides", "orc_core.h",
     "double sg = ((dk > 0) == (s == 1)) ? 1.0 : -1.0;", "double sg = (dk > 0) ? 1.0 : -1.0;",
     [(P.test_interior_face_fluxes_closed_form, (1,))]),
    ("terrain not decaying to a flat top", "orc_core.h",
     "zeta + orc_terrain_height(m, x, y) * (1.0 - zeta / m->Lz)", "zeta + orc_terrain_height(m, x, y)",
     [(P.test_terrain_following_map, (P.CURVED[0],))]),
    ("Lax-Friedrichs dissipation with the wrong sign", "orc_imex.c",
     "+ 0.5 * lam * an * (qm[fl] - qpv[fl]);", "- 0.5 * lam * an * (qm[fl] - qpv[fl]);",
     [(I.test_lax_friedrichs_upwind_closed_form, (1,))]),
    ("gravity work with the wrong sign", "orc_imex.c",
     "loc[4 * n3 + i] += wd * (-b->g * r * v[2]) * ps[i];", "loc[4 * n3 + i] += wd * (b->g * r * v[2]) * ps[i];",
     [(I.test_linear_density_constant_velocity, ())]),
    ("slip wall reflecting half the normal velocity", "orc_imex.c",
     "vp[d] = vm[d] - 2.0 * un * nh[d];", "vp[d] = vm[d] - un * nh[d];",
     [(I.test_mass_conservation_of_explicit_tendency, ())]),
    ("own velocity on both sides of the momentum flux", "orc_imex.c",
     "double qpv[5] = {rp, rp * vp[0], rp * vp[1], rp * vp[2], rp * kp};",
     "double qpv[5] = {rp, rp * vm[0], rp * vm[1], rp * vm[2], rp * kp};",
     [(I.test_explicit_momentum_and_energy_budgets, ())]),
    ("far-field wind along y", "orc_imex.c",
     "vp[0] = b->ubar; vp[1] = 0.0; vp[2] = 0.0;", "vp[0] = 0.0; vp[1] = b->ubar; vp[2] = 0.0;",
     [(I.test_far_field_free_stream, ())]),
    ("far-field ghost density from the interior trace", "orc_imex.c",
     "rp = dotn(n3, rho_bar + c * n3, ps);", "rp = rm;",
     [(I.test_far_field_inflow_mass_budget, ())]),
    ("earlier implicit stage terms weighted by the explicit tableau", "orc_imex.c",
     "Fs[i] += dt * (A[l * s + mm] * E[N + i] + At[l * s + mm] * E[5 * N + i]);",
     "Fs[i] += dt * (A[l * s + mm] * E[N + i] + A[l * s + mm] * E[5 * N + i]);",
     [(I.test_imex_euler_acoustics_closed_form, ())]),
    ("kinetic energy without the 1/2", "orc_imex.c",
     "double f = 0.5 * r * (v0 * v0 + v1 * v1 + v2 * v2) * G.wdet[qp];",
     "double f = r * (v0 * v0 + v1 * v1 + v2 * v2) * G.wdet[qp];",
     [(I.test_kinetic_mass_closed_form, (dict(terrain=0),))]),
    ("buoyancy of the stage with the wrong sign", "orc_imex.c",
     "orc_apply_M(m, -b->g * al, t1, t2);", "orc_apply_M(m, b->g * al, t1, t2);",
     [(I.test_buoyancy_initial_acceleration, (False,))]),
    ("hanging-face points of a base cell ignoring the child's position", "orc_core.h",
     "xi[k] = (double)s; xi[t1] = 0.5 * (sg1 + T->gq[i]);", "xi[k] = (double)s; xi[t1] = 0.5 * T->gq[i];",
     [(NC.test_B_reproduces_gradient_of_linear_fields, (2,))]),
    ("child's face normal not reversed on the base side", "orc_core.h",
     "nA[3 * p + d] = -nAc[3 * (i + q * j) + d];", "nA[3 * p + d] = nAc[3 * (i + q * j) + d];",
     [(NC.test_hanging_fluxes_cancel, ())]),
    ("child nodes all in the parent's first octant", "orc_core.h",
     "double xi[3] = {0.5 * (f[0] % 2 + T->gll[a]),", "double xi[3] = {0.5 * (T->gll[a]),",
     [(NC.test_cells_partition_the_domain, (NC.HILL,))]),
    ("children numbered y fastest", "orc_core.h",
     "return base_cells(m) + f[0] + fd[0] * (f[1] + fd[1] * f[2]);",
     "return base_cells(m) + f[1] + fd[1] * (f[0] + fd[0] * f[2]);",
     [(NC.test_fully_refined_mesh_is_the_conforming_fine_mesh, ())]),
    ("hanging C flux with the own kappa on both sides", "orc.c",
     "double flux = 0.5 * (kf * dotn(n3, kc, ps) * vm + kf * dotn(n3, pk + o, pn) * vp);",
     "double flux = 0.5 * (kf * dotn(n3, kc, ps) * vm + kf * dotn(n3, kc, ps) * vp);",
     [(NC.test_hanging_fluxes_cancel, ())]),
    ("hanging Lax-Friedrichs dissipation with the wrong sign", "orc_imex.c",
     "double F = 0.5 * (qm[fl] * unm + qn[fl] * unp) + 0.5 * lam * an * (qm[fl] - qn[fl]);",
     "double F = 0.5 * (qm[fl] * unm + qn[fl] * unp) - 0.5 * lam * an * (qm[fl] - qn[fl]);",
     [(NC.test_explicit_upwinds_a_density_jump_across_hanging_faces, ())]),
    ("velocity recovery with the wrong sign", "orc_imex.c",
     "ul[i] = W[i] - t2[i];", "ul[i] = W[i] + t2[i];",
     [(I.test_buoyancy_initial_acceleration, (False,)), (I.test_acoustic_standing_wave_closed_form, ())]),
]

PY_MUTANTS = [
    ("convolution taps in (x, y, z) order", "W[:, :, dz, dy, dx], patch)", "W[:, :, dx, dy, dz], patch)",
     [(TL.test_conv_matches_loop_definition, ())]),
    ("weight gradient of the flipped tap", 'gW[:, :, dz, dy, dx] = np.einsum("ozyx,izyx->oi", gy, patch)',
     'gW[:, :, 2 - dz, 2 - dy, 2 - dx] = np.einsum("ozyx,izyx->oi", gy, patch)',
     [(TL.test_backward_matches_finite_differences, ())]),
    ("ReLU after the last layer too", "h = np.maximum(z, 0.0) if i + 1 < len(params) else z",
     "h = np.maximum(z, 0.0)", [(TL.test_network_matches_torch_autograd, ())]),
    ("loss gradient without the factor 2", "gout = (2.0 * s[k] / nx2 / B * e)[None]",
     "gout = (s[k] / nx2 / B * e)[None]", [(TL.test_backward_matches_finite_differences, ())]),
    ("bf16 rounding half up", "rnd = ((u >> 16) & 1) + 0x7FFF", "rnd = 0x8000",
     [(TL.test_bf16_rounding, ())]),
    ("diagonal channel not normalised", "np.log(d / d.mean())", "np.log(d)",
     [(TL.test_features_normalisation, ())]),
    ("Adam without bias correction", "mh = m / (1.0 - b1 ** t)", "mh = m",
     [(TL.test_adam_closed_form, ())]),
    ("node index with a and c swapped", "cell * n ** 3 + a + n * b + n * n * c",
     "cell * n ** 3 + c + n * b + n * n * a", [(TL.test_grid_map_follows_the_mesh, ())]),
]


def _plant(text, old, new, name):
    assert text.count(old) == 1, "%s: the text to replace must occur once" % name
    return text.replace(old, new)


def _fails(pins):
    for pin, args in pins:
        try:
            pin(*args)
        except AssertionError:
            return True
    return False


@pytest.fixture(scope="module")
def c_sources(tmp_path_factory):
    base = tmp_path_factory.mktemp("oracle_src")
    for f in ("orc.c", "orc_imex.c", "orc_core.h"):
        shutil.copy(os.path.join(ORACLE, f), base / f)
    return base


@pytest.mark.parametrize("case", C_MUTANTS, ids=[c[0] for c in C_MUTANTS])
def test_planted_mistake_in_c_oracle_fails_a_pin(case, c_sources, tmp_path, monkeypatch):
    name, fname, old, new, pins = case
    for f in ("orc.c", "orc_imex.c", "orc_core.h"):
        shutil.copy(c_sources / f, tmp_path / f)
    path = tmp_path / fname
    path.write_text(_plant(path.read_text(), old, new, name))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=gnu99", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                    str(tmp_path / "orc.c"), str(tmp_path / "orc_imex.c"), "-lm"], check=True)
    O.lib()  # the real oracle is built and loaded first; the mutant replaces it for this test only
    monkeypatch.setattr(O, "_lib", ctypes.CDLL(str(lib)))
    assert _fails(pins), "planted mistake not caught: " + name


@pytest.mark.parametrize("case", PY_MUTANTS, ids=[c[0] for c in PY_MUTANTS])
def test_planted_mistake_in_network_oracle_fails_a_pin(case, monkeypatch):
    name, old, new, pins = case
    src = _plant(open(NL.__file__).read(), old, new, name)
    mod = types.ModuleType("oracle_learned_mutant")
    exec(compile(src, "<mutant of oracle/learned.py>", "exec"), mod.__dict__)
    for attr, val in vars(mod).items():
        if isinstance(val, types.FunctionType):
            monkeypatch.setattr(NL, attr, val)
    assert _fails(pins), "planted mistake not caught: " + name


def test_unmutated_pins_pass():
    """The same pins pass on the real oracle (so a failure above is the
    planted mistake's doing)."""
    for _, _, _, _, pins in C_MUTANTS:
        if not any(p is I.test_acoustic_standing_wave_closed_form for p, _ in pins):
            assert not _fails(pins)
    for _, _, _, pins in PY_MUTANTS:
        assert not _fails(pins)
