"""Planted mistakes in the oracle, on the CPU: each mutant is the oracle with one
plausible error (a wrong index rule, sign, operand, weight, layout or dropped
term), and the pins of ``test_oracle_pins.py`` listed beside it must fail on it.

C mutants are one textual change of ``oracle/l2x_oracle.c`` compiled into a
temporary library that the oracle loads instead of its own; Python mutants are
one change of ``oracle/__init__.py`` executed as a module of their own.  The
control cases run every detector on unchanged copies through the same harness,
so a detector failing on a mutant is the mutant's doing.  Nothing here touches
the oracle's files.
"""
import os
import subprocess
import sys
import types

import pytest

import oracle
import test_oracle_pins as pins

_ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))

DETECTORS = {
    "pairs2": lambda: pins.test_candidate_pairs_match_bruteforce_on_dyadic_input(2),
    "pairs3": lambda: pins.test_candidate_pairs_match_bruteforce_on_dyadic_input(3),
    "rows2": lambda: pins.test_row_sums_and_total_volume("disk2d"),
    "rows3": lambda: pins.test_row_sums_and_total_volume("beam16"),
    "exact2": lambda: pins.test_pair_blocks_match_exact_rational("disk2d_small", 5),
    "exact3": lambda: pins.test_pair_blocks_match_exact_rational("beam16", 230),
    "textbook2": lambda: pins.test_element_inside_one_cell_is_textbook(2),
    "textbook3": lambda: pins.test_element_inside_one_cell_is_textbook(3),
    "columns": pins.test_column_sums_of_covered_fluid_nodes,
    "affine2": lambda: pins.test_affine_fields_are_reproduced("disk2d"),
    "affine3": lambda: pins.test_affine_fields_are_reproduced("beam16"),
    "golden": pins.test_golden_2d_exact_block,
    "mass": pins.test_mass_matrix_matches_exact_quadrature,
    "adjoint2": lambda: pins.test_force_transfer_is_the_adjoint("disk2d"),
    "dual_exact2": lambda: pins.test_dual_blocks_match_exact_rational("disk2d_small", 5),
    "dual_rows3": lambda: pins.test_dual_rows_sum_to_the_lumped_mass("beam16"),
    "dual_affine3": lambda: pins.test_dual_projection_reproduces_affine_fields("beam16"),
    "picard": pins.test_picard_norms_and_criteria_closed_form,
    "solve_cg": lambda: pins.test_mass_solves_satisfy_the_defining_equation("cg"),
    "s_pairs2": lambda: pins.test_stretched_candidate_pairs_match_bruteforce(2),
    "s_pairs3": lambda: pins.test_stretched_candidate_pairs_match_bruteforce(3),
    "s_rows2": lambda: pins.test_stretched_row_sums_and_affine_reproduction("disk2d_s"),
    "s_rows3": lambda: pins.test_stretched_row_sums_and_affine_reproduction("beam16s"),
}

# (name, text in l2x_oracle.c, replacement, detectors that must catch it)
C_MUTANTS = [
    ("bbox_misses_last_vertex",
     "    for (int v = 0; v <= dim; ++v) {\n        const double* p = X + (int64_t)E[e * (dim + 1) + v] * dim;",
     "    for (int v = 0; v < dim; ++v) {\n        const double* p = X + (int64_t)E[e * (dim + 1) + v] * dim;",
     ["pairs2", "pairs3"]),
    ("upper_index_keeps_cell_beyond_grid_line",
     "ihi[k] = (int64_t)ceil(qhi) - 1;", "ihi[k] = (int64_t)floor(qhi);", ["pairs2", "pairs3"]),
    ("lower_index_keeps_cell_below_grid_line",
     "ilo[k] = (int64_t)floor(qlo);", "ilo[k] = (int64_t)ceil(qlo) - 1;", ["pairs2", "pairs3"]),
    ("linear_cell_index_transposed",
     "pair_cell[p] = ix + ncell[0] * (iy + ncell[1] * iz);",
     "pair_cell[p] = iy + ncell[1] * (ix + ncell[0] * iz);", ["pairs2", "pairs3"]),
    ("half_space_sign",
     "return side == 0 ? p[k] - c : c - p[k];", "return side == 0 ? p[k] - c : p[k] - c;", ["rows2", "rows3"]),
    ("cut_parameter_from_wrong_end",
     "double t = sp / (sp - sq);", "double t = sq / (sq - sp);", ["rows2", "rows3"]),
    ("quadrilateral_split_wrong_triangle",
     "set_pt(&T, 0, S->v[a], 2); set_pt(&T, 1, pbc, 2); set_pt(&T, 2, pac, 2);",
     "set_pt(&T, 0, S->v[b], 2); set_pt(&T, 1, pbc, 2); set_pt(&T, 2, pac, 2);", ["rows2", "exact2"]),
    ("prism_split_wrong_tetrahedron",
     "{0, 4, 5, 3}}", "{0, 4, 5, 2}}", ["rows3"]),
    ("three_point_weights_swapped",
     "wz[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0}", "wz[3] = {8.0 / 9.0, 5.0 / 9.0, 8.0 / 9.0}",
     ["textbook2", "rows2"]),
    ("four_point_weights_swapped",
     "wz[4] = {w2, w1, w1, w2}", "wz[4] = {w1, w2, w2, w1}", ["textbook3", "rows3"]),
    ("collapsed_map_jacobian",
     "double jac = dim == 3 ? u * u * v * D : u * D;", "double jac = dim == 3 ? u * v * v * D : u * D;",
     ["textbook3", "rows3"]),
    ("collapsed_map_directions_swapped",
     "x[j] = p[0][j] + u * (A[j] + v * (B[j] + w * C[j]));",
     "x[j] = p[0][j] + u * (A[j] + w * (B[j] + v * C[j]));", ["textbook2", "textbook3"]),
    ("barycentric_row_and_column_transposed",
     "double s = Minv[a][dim];", "double s = Minv[dim][a];", ["textbook2", "textbook3"]),
    ("barycentric_map_coordinates_permuted",
     "A[r][c] = (r < dim) ? V[c][r] : 1.0;", "A[r][c] = (r < dim) ? V[c][(r + 1) % dim] : 1.0;",
     ["textbook2", "textbook3"]),
    ("corner_bit_reversed",
     "psi *= ((b >> j) & 1) ? t[j] : 1.0 - t[j];", "psi *= ((b >> j) & 1) ? 1.0 - t[j] : t[j];",
     ["textbook2", "exact2", "affine3"]),
    ("block_layout_transposed",
     "block[a * nb + b] += f * lam[a] * psi;", "block[b * na + a] += f * lam[a] * psi;",
     ["textbook2", "textbook3"]),
    ("cell_origin_off_by_one",
     "clo[k] = origin[k] + (double)ci[k] * h_uniform[k];",
     "clo[k] = origin[k] + (double)(ci[k] + 1) * h_uniform[k];", ["rows2", "rows3"]),
    ("cell_decode_y_strides_swapped",
     "ci[1] = (cell / ncell[0]) % ncell[1];", "ci[1] = (cell / ncell[1]) % ncell[0];", ["rows3", "affine3"]),
    ("cell_decode_z_stride",
     "if (dim == 3) ci[2] = cell / (ncell[0] * ncell[1]);", "if (dim == 3) ci[2] = cell / (ncell[0] * ncell[2]);",
     ["rows3", "affine3"]),
    ("cut_point_not_on_the_plane",
     "    r[k] = c;\n", "    r[k] = p[k];\n", ["rows2", "rows3"]),
    ("stretched_upper_cell_not_strict",
     "ihi[k] = count_lt(axis[k], ncell[k] + 1, hi[k]) - 1;", "ihi[k] = count_le(axis[k], ncell[k] + 1, hi[k]) - 1;",
     ["s_pairs2", "s_pairs3"]),
    ("stretched_lower_cell_strict",
     "ilo[k] = count_le(axis[k], ncell[k] + 1, lo[k]) - 1;", "ilo[k] = count_lt(axis[k], ncell[k] + 1, lo[k]) - 1;",
     ["s_pairs2", "s_pairs3"]),
    ("stretched_first_width_for_every_cell",
     "h[k] = axis[k][ci[k] + 1] - axis[k][ci[k]];", "h[k] = axis[k][1] - axis[k][0];", ["s_rows2", "s_rows3"]),
]

# (name, text in oracle/__init__.py, replacement, detectors)
PY_MUTANTS = [
    ("mass_normalisation",
     "loc = (np.ones((na, na)) + np.eye(na)) / ((d + 1) * (d + 2))",
     "loc = (np.ones((na, na)) + np.eye(na)) / ((d + 1) * (d + 1))", ["mass"]),
    ("mass_delta_on_the_antidiagonal",
     "loc = (np.ones((na, na)) + np.eye(na)) / ((d + 1) * (d + 2))",
     "loc = (np.ones((na, na)) + np.eye(na)[::-1]) / ((d + 1) * (d + 2))", ["mass"]),
    ("element_volume_factor",
     "return np.abs(np.linalg.det(J)) / (2.0 if d == 2 else 6.0)",
     "return np.abs(np.linalg.det(J)) / (2.0 if d == 2 else 3.0)", ["rows3", "mass"]),
    ("corner_bits_in_reverse_axis_order",
     "idx = [ci[k] + ((b >> k) & 1) for k in range(d)]",
     "idx = [ci[k] + ((b >> (d - 1 - k)) & 1) for k in range(d)]", ["golden", "columns", "affine2"]),
    ("node_strides_swapped",
     "out[:, b] = idx[0] + nn[0] * (idx[1] + nn[1] * idx[2])",
     "out[:, b] = idx[0] + nn[1] * (idx[1] + nn[0] * idx[2])", ["affine3"]),
    ("zero_volume_pairs_kept",
     "keep = vols > 0.0", "keep = vols >= 0.0", ["golden"]),
    ("dual_weight",
     "return (d + 2) * blocks - blocks.sum(axis=1, keepdims=True)",
     "return (d + 1) * blocks - blocks.sum(axis=1, keepdims=True)", ["dual_exact2", "dual_affine3"]),
    ("lumped_mass_factor",
     "np.add.at(diag, E[:, a], vol / (d + 1))", "np.add.at(diag, E[:, a], vol / (d + 2))",
     ["dual_rows3", "dual_affine3"]),
    ("force_modes_swapped",
     'Z = self.solve_S(F) if mode == "dual" else F', 'Z = F if mode == "dual" else self.solve_S(F)', ["adjoint2"]),
    ("velocity_fields_of_the_wrong_grid",
     "Y = np.stack([self.B[g] @ np.asarray(fields[g], dtype=np.float64)",
     "Y = np.stack([self.B[g] @ np.asarray(fields[-1 - g], dtype=np.float64)", ["affine3"]),
    ("norm_without_absolute_value",
     "return float(np.max(np.abs(a - b))), float(np.max(np.abs(a)))",
     "return float(np.max(np.abs(a - b))), float(np.max(a))", ["picard"]),
    ("absolute_criterion_not_strict",
     "return d_norm < eps_abs or", "return d_norm <= eps_abs or", ["picard"]),
    ("force_scale_dropped",
     "return [scale * (self.B[g].T @ Z[:, g]) for g in range(len(self.B))]",
     "return [(self.B[g].T @ Z[:, g]) for g in range(len(self.B))]", ["adjoint2"]),
    ("cg_step_length",
     "alpha = rr / (p @ q)", "alpha = rr / (q @ q)", ["solve_cg"]),
    ("cg_direction_update_inverted",
     "p = r + (rr_new / rr) * p", "p = r + (rr / rr_new) * p", ["solve_cg"]),
]


def _compile_c(tmp_path, old=None, new=None):
    with open(os.path.join(_ORACLE_DIR, "l2x_oracle.c")) as f:
        src = f.read()
    if old is not None:
        assert src.count(old) == 1, f"mutation site not unique: {old!r}"
        src = src.replace(old, new)
    c = tmp_path / "l2x_oracle_variant.c"
    c.write_text(src)
    so = tmp_path / "liborc_variant.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", "-o", str(so),
                           str(c), "-lm"])
    return str(so)


def _use_c_library(monkeypatch, so):
    monkeypatch.setattr(oracle, "_LIB_PATH", so)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: so)


def _use_py_module(monkeypatch, old=None, new=None):
    path = oracle.__file__
    with open(path) as f:
        src = f.read()
    if old is not None:
        assert src.count(old) == 1, f"mutation site not unique: {old!r}"
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_variant")
    mod.__file__ = path
    monkeypatch.setitem(sys.modules, "oracle_variant", mod)
    exec(compile(src, path, "exec"), mod.__dict__)
    monkeypatch.setattr(pins, "oracle", mod)


def _caught(names):
    for n in names:
        try:
            DETECTORS[n]()
        except Exception:
            return n
    return None


def test_detectors_pass_on_unchanged_copies(tmp_path, monkeypatch):
    """Control: the harness itself leaves every detector passing."""
    _use_c_library(monkeypatch, _compile_c(tmp_path))
    _use_py_module(monkeypatch)
    for name, f in DETECTORS.items():
        f()


@pytest.mark.parametrize("name,old,new,detectors", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_c_mutant_is_caught(name, old, new, detectors, tmp_path, monkeypatch):
    _use_c_library(monkeypatch, _compile_c(tmp_path, old, new))
    assert _caught(detectors) is not None, f"no pin caught the planted mistake {name}"


@pytest.mark.parametrize("name,old,new,detectors", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_python_mutant_is_caught(name, old, new, detectors, monkeypatch):
    _use_py_module(monkeypatch, old, new)
    assert _caught(detectors) is not None, f"no pin caught the planted mistake {name}"
