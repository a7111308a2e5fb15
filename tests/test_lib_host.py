"""Host-side checks of librsrs (no GPU needed): symbols, tree parity with the oracle, argument errors."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle.tree import Schedule as OSchedule
from oracle.tree import Tree as OTree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2311_01451_gb300 as pkg

    return pkg


def test_every_declared_symbol_is_exported(R):
    hdr = open(os.path.join(ROOT, "include", "rsrs.h")).read()
    declared = set(re.findall(r"\b(rsrs_[a-z0-9_]+)\s*\(", hdr)) - {"rsrs_matvec_fn"}
    lib = R.lib()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(R.rsrs.EXPORTS) <= declared


@pytest.mark.parametrize("case", ["grid2d", "rand2d", "rand3d", "clustered2d", "collinear2d", "coincident2d",
                                  "single", "outside_unit3d", "planar3d"])
def test_tree_and_schedule_match_oracle(R, case):
    """Same tree, order and schedule as the oracle's, including degenerate geometry: points on a
    line or a plane (empty children are never made), 100 coincident points (subdivision stops at the
    2^20 binning grid's depth), one point (a root-only tree), and points outside the unit cube (the
    root is their bounding cube)."""
    if case == "grid2d":
        pts, leaf, k = W.grid_points_2d(64), 64, 32
    elif case == "rand2d":
        pts, leaf, k = W.uniform_points(20000, 2, W.rng_for(96, 0, 0)), 64, 24
    elif case == "rand3d":
        pts, leaf, k = W.uniform_points(6000, 3, W.rng_for(96, 1, 0)), 32, 16
    elif case == "clustered2d":
        pts = np.vstack([W.uniform_points(3000, 2, W.rng_for(96, 2, 0)) * 0.03 + 0.5,
                         W.uniform_points(2000, 2, W.rng_for(96, 3, 0))])
        leaf, k = 20, 8
    elif case == "collinear2d":
        pts = np.stack([W.uniform_points(3000, 1, W.rng_for(96, 4, 0))[:, 0], np.full(3000, 0.25)], 1)
        leaf, k = 24, 8
    elif case == "coincident2d":
        pts = np.vstack([np.full((100, 2), 0.3), W.uniform_points(400, 2, W.rng_for(96, 5, 0))])
        leaf, k = 16, 8
    elif case == "single":
        pts, leaf, k = np.array([[0.5, 0.5]]), 16, 8
    elif case == "outside_unit3d":
        pts, leaf, k = W.uniform_points(3000, 3, W.rng_for(96, 6, 0)) * 8.0 - 3.0, 32, 12
    else:
        pts = np.hstack([W.uniform_points(4000, 2, W.rng_for(96, 7, 0)), np.full((4000, 1), 0.5)])
        leaf, k = 32, 12
    t = R.Tree(pts, leaf)
    ot = OTree(pts, leaf)
    osc = OSchedule(ot, k)
    info = t.info(k)
    assert info.depth == ot.depth
    assert np.array_equal(t.perm(), ot.perm)
    assert info.s_req == osc.s_req and info.root_size == osc.root_size and info.max_l == osc.max_l
    assert info.s_req_mixed >= info.s_req
    sch = t.schedule(k)
    ref = np.array([[st["level"], st["colour"], st["b"], st["n"], st["box"].first_pos] for st in osc.steps])
    assert np.array_equal(sch[:, [0, 1, 3, 4, 5]], ref.reshape(-1, 5))
    if case == "coincident2d":
        assert info.depth == 20
    if case == "single":
        assert info.n_compress == 0 and info.root_size == 1


def test_sample_bound_matches_paper(R):
    t = R.Tree(W.grid_points_2d(284), 160)
    assert t.info(40).s_req == 1520  # 37k + p, Exp. 1


def test_invalid_arguments(R):
    lib = R.lib()
    h = C.c_void_p()
    assert lib.rsrs_tree_build(None, 10, 2, 4, C.byref(h)) == 1
    pts = np.zeros((10, 4))
    assert lib.rsrs_tree_build(pts.ctypes.data_as(C.c_void_p), 10, 4, 4, C.byref(h)) == 1
    bad = W.uniform_points(10, 2, W.rng_for(97, 0, 0))
    bad[3, 0] = np.nan
    assert lib.rsrs_tree_build(bad.ctypes.data_as(C.c_void_p), 10, 2, 4, C.byref(h)) == 1
    assert lib.rsrs_status_string(2) == b"sample count below the bound s_req"


def test_undersampled_rejected_before_device_work(R):
    t = R.Tree(W.grid_points_2d(64), 64)
    s_req = t.info(32).s_req
    with pytest.raises(R.RSRSError) as e:
        R.Factor(t, R.RSRS_OP_LOG2D, 32, 400, shift=1.0, scale=1 / 4096)  # the literal s of the 64x64 workload
    assert e.value.name == "RSRS_E_UNDERSAMPLED" and s_req > 400
    with pytest.raises(R.RSRSError) as e:
        R.Factor(t, R.RSRS_OP_INVR3D, 32, s_req)  # 3D kernel on 2D points
    assert e.value.name == "RSRS_E_INVAL"


@pytest.mark.parametrize("tune", [{"sample_tile": 8}, {"cpqr_cluster": 3}, {"cpqr_threads": 100},
                                  {"residual_split": 17}, {"sample_tile": -1}])
def test_tune_values_validated_before_device_work(R, tune):
    t = R.Tree(W.grid_points_2d(64), 64)
    with pytest.raises(R.RSRSError) as e:
        R.Factor(t, R.RSRS_OP_LOG2D, 32, t.info(32).s_req, shift=1.0, scale=1 / 4096, tune=tune)
    assert e.value.name == "RSRS_E_INVAL"


def test_autotune_cache_hit_needs_no_device(R, tmp_path):
    """A cache line for the problem's key is returned as is, without a build (so also here)."""
    t = R.Tree(W.grid_points_2d(64), 64)
    s = t.info(32).s_req_mixed
    cache = tmp_path / "tune.txt"
    # the key starts with the device name; without a device the library reports "unknown"
    name = "unknown"
    try:
        import torch
        if torch.cuda.is_available():
            name = torch.cuda.get_device_name(0).replace(" ", "_")
    except ImportError:
        pass
    cache.write_text(f"{name} {R.RSRS_OP_LOG2D} 1 4096 2 32 {s} {R.RSRS_PREC_MIXED} 2 4 512 8\n")
    tune, rep = R.autotune(t, R.RSRS_OP_LOG2D, 32, s, 1.0, 1 / 4096, cache=str(cache))
    assert rep["from_cache"] and rep["candidates"] == 0
    assert tune == {"sample_tile": 2, "cpqr_cluster": 4, "cpqr_threads": 512, "residual_split": 8}


def test_autotune_validates_before_device_work(R):
    t = R.Tree(W.grid_points_2d(64), 64)
    s = t.info(32).s_req_mixed
    with pytest.raises(R.RSRSError) as e:
        R.autotune(t, R.RSRS_OP_LOG2D, 32, s, 1.0, 1 / 4096, tune={"cpqr_threads": 7})
    assert e.value.name == "RSRS_E_INVAL"
    lib = R.lib()
    assert lib.rsrs_autotune(1, None, None, 32, s, None, 1, None, None, None, None) == 1


STRUCTS = {"Operator": "rsrs_operator", "Tune": "rsrs_tune_t", "TuneReport": "rsrs_tune_report",
           "Options": "rsrs_options", "TreeInfo": "rsrs_tree_info_t", "Stats": "rsrs_stats",
           "RefineReport": "rsrs_refine_report", "BoxView": "rsrs_box_view"}


def test_binding_struct_layouts_match_the_header(R, tmp_path):
    """Every struct the binding passes through the C ABI has the header's size and field offsets
    (a C program compiled against include/rsrs.h prints them; no device work)."""
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rsrs.h"', "int main(void) {"]
    want = []
    for py, c in STRUCTS.items():
        cls = getattr(R.rsrs, py)
        lines.append(f'  printf("%zu\\n", sizeof({c}));')
        want.append(C.sizeof(cls))
        for name, *_ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({c}, {name}));')
            want.append(getattr(cls, name).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want


@pytest.mark.parametrize("mode", [-1, 4])
def test_residual_arithmetic_validated_before_device_work(R, mode):
    t = R.Tree(W.grid_points_2d(64), 64)
    with pytest.raises(R.RSRSError) as e:
        R.Factor(t, R.RSRS_OP_LOG2D, 32, t.info(32).s_req, shift=1.0, scale=1 / 4096, residual=mode)
    assert e.value.name == "RSRS_E_INVAL"


@pytest.mark.parametrize("kernel,precision", [(4, 0), (-1, 0), (3, 1)])
def test_sample_kernel_validated_before_device_work(R, kernel, precision):
    """sample_kernel out of range, and the Ozaki FP64 sampling (3) asked of a mixed build, are
    refused with RSRS_E_INVAL before any device work."""
    t = R.Tree(W.grid_points_2d(64), 64)
    with pytest.raises(R.RSRSError) as e:
        R.Factor(t, R.RSRS_OP_LOG2D, 32, t.info(32).s_req_mixed, shift=1.0, scale=1 / 4096, precision=precision,
                 sample_kernel=kernel)
    assert e.value.name == "RSRS_E_INVAL"
