"""Planted mistakes in the oracle: is every pin able to catch a plausible slip?

Each mutant is a copy of one oracle module, compiled from its source with one small textual change
(a flipped sign, a dropped term, a transposed or swapped operand, an off-by-one index, a wrong
threshold), swapped in for the real module's functions for the length of one test.  The oracle's
own pins (the tests in test_oracle_*.py: closed forms, exactness on matrices with exactly low-rank
off-diagonal blocks, brute force against dense LU, library routines, invariants) then run against
it, and at least one of them must fail.  The control case compiles the unchanged source the same
way and must pass every pin, so a failure is the planted mistake's and not the harness's.

Everything here runs on the CPU; nothing is planted in the CUDA path.
"""
import os
import sys
import types
from dataclasses import dataclass

import numpy as np
import pytest

import oracle.linalg
import oracle.operators
import oracle.refine
import oracle.rsrs
import oracle.tree
import test_golden_exp1 as tgold
import test_oracle_gmres as tg
import test_oracle_linalg as tl
import test_oracle_rsrs as tr
import test_oracle_tree as tt
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RSRS_PINS = [tr.test_exact_h2_matrix_is_reproduced_to_rounding, tr.test_apply_solve_inverse_and_adjoints,
             tr.test_extraction_is_exact_when_far_field_vanishes, tr.test_sketch_pair_invariant]
LINALG_PINS = [tl.test_null_basis, tl.test_pinv_right_matches_svd_pinv, tl.test_cpqr_matches_lapack_pivoted_qr,
               tl.test_cpqr_exact_low_rank_truncation, tl.test_cpqr_tie_goes_to_lowest_index,
               tl.test_cpqr_rows_below_the_absolute_floor_are_dependent]
OPS_PINS = [tl.test_kernel_entries_scalar_formula, tl.test_kernel_operator_is_symmetric_and_samples_match_dense,
            tl.test_stencil7_closed_forms]
TREE_PINS = [lambda: tt.test_tree_partition_and_balance(lambda: W.grid_points_2d(32), 16),
             lambda: tt.test_tree_partition_and_balance(
                 lambda: np.vstack([W.uniform_points(1500, 2, W.rng_for(93, 0, 0)) * 0.05,
                                    W.uniform_points(500, 2, W.rng_for(93, 1, 0))]), 12),
             tt.test_uniform_grid_neighbour_counts,
             lambda: tt.test_colouring_is_conflict_free(16, 4),
             tt.test_uniform_3d_sample_count, tt.test_sizes_and_root,
             lambda: tgold.test_oracle_sample_count_matches_table(tgold.ROWS[0], 40)]
GMRES_PINS = [lambda: tg.test_terminates_after_distinct_eigenvalue_count(3), tg.test_exact_preconditioner_one_iteration,
              tg.test_estimates_monotone_and_true_residual, tg.test_restarts_converge_to_dense_solution,
              tg.test_preconditioned_matches_refinement_fixed_point]
REFINE_PINS = [tr.test_refinement_reaches_dense_solution, tr.test_refinement_stopping_rule_is_relative] + GMRES_PINS

PINS = {"rsrs": RSRS_PINS, "linalg": LINALG_PINS, "operators": OPS_PINS, "tree": TREE_PINS,
        "refine": REFINE_PINS}
MODULES = {"rsrs": oracle.rsrs, "linalg": oracle.linalg, "operators": oracle.operators, "tree": oracle.tree,
           "refine": oracle.refine}


@dataclass
class Mutant:
    name: str
    module: str
    old: str
    new: str


MUTANTS = [
    # Algorithm 1 (oracle/rsrs.py)
    Mutant("schur_sign", "rsrs", "Y[S] -= LcS @ YR", "Y[S] += LcS @ YR"),
    Mutant("schur_drops_neighbour_term", "rsrs", "Om[R] += UcS @ Om[S] + UcN @ Om[Nact]", "Om[R] += UcS @ Om[S]"),
    Mutant("e_update_missing_on_z", "rsrs", "            Z[R] -= T.T @ Z[S]\n", ""),
    Mutant("e_update_missing_on_y", "rsrs", "            Y[R] -= T.T @ Y[S]\n", ""),
    Mutant("schur_z_neighbour_sign", "rsrs", "Z[Nact] -= UcN.T @ ZR", "Z[Nact] += UcN.T @ ZR"),
    Mutant("redundant_indices_stay_active", "rsrs", "act[box.id] = _tree_sorted(S, tree.pos)",
           "act[box.id] = _tree_sorted(Bact, tree.pos)"),
    Mutant("f_update_wrong_sketch", "rsrs", "Ps[S] += T @ Ps[R]", "Ps[S] += T @ Om[R]"),
    Mutant("nullify_z_with_omega", "rsrs", "Zp = Z[Bact] @ la.null(Ps[BN])", "Zp = Z[Bact] @ la.null(Om[BN])"),
    Mutant("id_of_y_side_only", "rsrs", "la.cpqr_id(np.hstack([Yp, Zp])", "la.cpqr_id(np.hstack([Yp, Yp])"),
    Mutant("extract_z_with_omega", "rsrs", "Xz = la.pinv_right(Z[R], Ps[BN])", "Xz = la.pinv_right(Z[R], Om[BN])"),
    Mutant("extract_neighbour_off_by_one", "rsrs", "cN = np.arange(b, l)", "cN = np.arange(b - 1, l - 1)"),
    Mutant("lc_untransposed_solve", "rsrs", "LcS = la.lu_solve(f, XSR.T, trans=1).T",
           "LcS = la.lu_solve(f, XSR.T, trans=0).T"),
    Mutant("root_from_psi", "rsrs", "fac.root_A = la.pinv_right(Y[Bt], Om[Bt])",
           "fac.root_A = la.pinv_right(Y[Bt], Ps[Bt])"),
    Mutant("upward_sweep_sign", "rsrs", "x[R] -= bf.T.T @ x[S]", "x[R] += bf.T.T @ x[S]"),
    Mutant("downward_sweep_sign", "rsrs", "x[S] -= bf.T @ x[R]", "x[S] += bf.T @ x[R]"),
    Mutant("diag_solve_adjoint_untransposed", "rsrs", "x[bf.R] = la.lu_solve(bf.lu, x[bf.R], trans=1 if adjoint else 0)",
           "x[bf.R] = la.lu_solve(bf.lu, x[bf.R], trans=0)"),
    Mutant("apply_adjoint_wrong_factor", "rsrs", "x[R] += bf.LcS.T @ x[S] + bf.LcN.T @ x[N]",
           "x[R] += bf.UcS @ x[S] + bf.UcN @ x[N]"),
    # building blocks (oracle/linalg.py)
    Mutant("null_leading_columns", "linalg", "return q[:, l:]", "return q[:, :s - l]"),
    Mutant("pinv_transposed_triangle", "linalg", "(y @ q).T, lower=False)", "(y @ q).T, lower=False, trans=1)"),
    Mutant("cpqr_norms_include_factored_rows", "linalg", "np.sum(a[j:, j:] ** 2, axis=0)",
           "np.sum(a[:, j:] ** 2, axis=0)"),
    Mutant("cpqr_tie_to_highest_index", "linalg", "cand[np.argmin(perm[j + cand])]",
           "cand[np.argmax(perm[j + cand])]"),
    Mutant("cpqr_t_columns_not_reordered", "linalg", "    t = t[:, order]\n", ""),
    Mutant("cpqr_floor_ignored", "linalg", "if best <= floor or", "if"),
    Mutant("householder_reflects_twice", "linalg", "a[j:, j:] -= 2.0 * np.outer", "a[j:, j:] -= 4.0 * np.outer"),
    Mutant("cpqr_pivot_smallest_norm", "linalg", "best = norms.max()", "best = norms.min()"),
    Mutant("cpqr_swap_forgets_perm", "linalg", "            perm[[j, p]] = perm[[p, j]]\n", ""),
    Mutant("cpqr_t_from_lower_triangle", "linalg",
           "t[:j0] = sla.solve_triangular(r11[:j0, :j0], r12[:j0], lower=False)",
           "t[:j0] = sla.solve_triangular(r11[:j0, :j0].T, r12[:j0], lower=True)"),
    Mutant("pinv_result_untransposed", "linalg", "return sla.solve_triangular(r, (y @ q).T, lower=False).T",
           "return sla.solve_triangular(r, (y @ q).T, lower=False)"),
    # matrices (oracle/operators.py)
    Mutant("log_of_r_squared", "operators", "k = np.log(r)", "k = np.log(r * r)"),
    Mutant("invr_squared", "operators", "k = 1.0 / r\n", "k = 1.0 / (r * r)\n"),
    Mutant("shift_replaced_by_scale", "operators", "idx] += self.shift", "idx] += self.scale"),
    Mutant("stencil_arithmetic_mean", "operators", "beta = 2.0 * bl * bh / (bl + bh)", "beta = 0.5 * (bl + bh)"),
    Mutant("stencil_wall_full_cell", "operators", "be = 2.0 * bb[tuple(e)]", "be = bb[tuple(e)]"),
    # geometry (oracle/tree.py)
    Mutant("neighbours_exclude_corners", "tree", "t = np.all((lo <= bhi[0]) & (blo[0] <= hi), axis=1)",
           "t = np.all((lo < bhi[0]) & (blo[0] < hi), axis=1)"),
    Mutant("colouring_checks_first_member_only", "tree", "for o in members[c.id]:", "for o in members[c.id][:1]:"),
    Mutant("sample_bound_without_k", "tree", "self.max_l + self.k + self.p", "self.max_l + self.p"),
    Mutant("sample_bound_without_p", "tree", "self.max_l + self.k + self.p", "self.max_l + self.k"),
    Mutant("position_map_not_inverted", "tree", "self.pos[self.perm] = np.arange(self.n)", "self.pos[:] = self.perm"),
    Mutant("balance_allows_two_levels", "tree", "deep = lvl >= a.level + 2", "deep = lvl >= a.level + 3"),
    # refinement and GMRES (oracle/refine.py)
    Mutant("refine_subtracts_correction", "refine", "x = x + rsrs.solve(fac, r)", "x = x - rsrs.solve(fac, r)"),
    Mutant("refine_residual_with_the_factor", "refine", "r = b - op.matvec(x)", "r = b - rsrs.apply(fac, x)"),
    Mutant("refine_stops_on_absolute_residual", "refine", "rel = np.linalg.norm(r) / bn", "rel = np.linalg.norm(r)"),
    Mutant("gmres_update_not_preconditioned", "refine", "x = x + precond(V[:, :k] @ y)", "x = x + V[:, :k] @ y"),
    Mutant("gmres_givens_sign", "refine", "g[k + 1], g[k] = -sn[k] * g[k], cs[k] * g[k]",
           "g[k + 1], g[k] = sn[k] * g[k], cs[k] * g[k]"),
    Mutant("gmres_no_orthogonalisation", "refine", "w = w - H[i, k] * V[:, i]", "w = w"),
    Mutant("gmres_left_rotation_stale", "refine", "H[i, k], H[i + 1, k] = cs[i] * a + sn[i] * c2, -sn[i] * a + cs[i] * c2",
           "H[i, k], H[i + 1, k] = cs[i] * a + sn[i] * c2, cs[i] * c2"),
]


# The ID's thresholds (oracle/rsrs.py) have pins of their own, too slow to run for every mutant above:
# a floor placed at the near field's 1e-10 (the accuracy pin) or dropped (the zero-far-field pin).
THRESHOLD_PINS = [tr.test_sparse_operator_boxes_have_no_far_field,
                  lambda: tr.test_id_thresholds_keep_the_far_field_rank(pytest.MonkeyPatch())]
THRESHOLD_MUTANTS = [
    Mutant("id_floor_at_1e-10_of_the_near_field", "rsrs", "floor = nullification_rounding(s) * np.sqrt(",
           "floor = 1e-10 * np.sqrt("),
    Mutant("id_floor_dropped", "rsrs", "floor = nullification_rounding(s) * np.sqrt(np.max(scale2))", "floor = 0.0"),
]


def _compile(module: str, old: str = "", new: str = "") -> types.ModuleType:
    """The oracle module ``module`` compiled from its source with ``old`` replaced by ``new``."""
    path = os.path.join(ROOT, "oracle", module + ".py")
    with open(path) as f:
        src = f.read()
    if old:
        assert src.count(old) == 1, f"{old!r} must occur once in oracle/{module}.py"
        src = src.replace(old, new)
    name = f"oracle._planted_{module}"
    mod = types.ModuleType(name)
    mod.__package__ = "oracle"
    mod.__file__ = path
    sys.modules[name] = mod  # dataclasses look their module up while the class body runs
    try:
        exec(compile(src, path, "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


def _swap_in(monkeypatch, module: str, mod: types.ModuleType):
    """Replace every function and class of the real module by the compiled copy's, wherever a
    module holds it by name (``from oracle.tree import Tree`` binds the class itself)."""
    real = MODULES[module]
    swap = {}
    for k, v in vars(mod).items():
        if isinstance(v, (types.FunctionType, type)) and getattr(v, "__module__", None) == mod.__name__:
            swap[id(getattr(real, k))] = v
    holders = list(MODULES.values()) + [tg, tgold, tl, tr, tt]
    for h in holders:
        for k, v in list(vars(h).items()):
            if id(v) in swap:
                monkeypatch.setattr(h, k, swap[id(v)])


def _failing_pins(pins):
    failed = []
    with np.errstate(all="ignore"):
        for pin in pins:
            try:
                pin()
            except Exception as e:  # an assertion, or a shape error the slip causes
                failed.append((getattr(pin, "__name__", "pin"), type(e).__name__))
    return failed


@pytest.mark.parametrize("module", sorted(PINS))
def test_unchanged_source_passes_every_pin(monkeypatch, module):
    _swap_in(monkeypatch, module, _compile(module))
    assert _failing_pins(PINS[module]) == []


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m.name for m in MUTANTS])
def test_planted_mistake_fails_a_pin(monkeypatch, mutant):
    _swap_in(monkeypatch, mutant.module, _compile(mutant.module, mutant.old, mutant.new))
    assert _failing_pins(PINS[mutant.module]), f"no pin of oracle/{mutant.module}.py catches {mutant.name}"


def test_unchanged_source_passes_the_threshold_pins(monkeypatch):
    _swap_in(monkeypatch, "rsrs", _compile("rsrs"))
    assert _failing_pins(THRESHOLD_PINS) == []


@pytest.mark.parametrize("mutant", THRESHOLD_MUTANTS, ids=[m.name for m in THRESHOLD_MUTANTS])
def test_planted_threshold_mistake_fails_a_pin(monkeypatch, mutant):
    _swap_in(monkeypatch, mutant.module, _compile(mutant.module, mutant.old, mutant.new))
    assert _failing_pins(THRESHOLD_PINS), f"no threshold pin catches {mutant.name}"


def test_every_oracle_module_is_covered():
    names = {os.path.splitext(f)[0] for f in os.listdir(os.path.join(ROOT, "oracle"))
             if f.endswith(".py") and f != "__init__.py"}
    assert names == set(PINS)
    assert all(sum(m.module == k for m in MUTANTS) >= 4 for k in PINS)
