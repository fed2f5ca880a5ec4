"""The C-ABI library loads and exports every entry point include/ucn.h
declares, and rejects malformed descriptors before touching the device
(these checks need no GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ucn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(ucn_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def ucn():
    from paper_2603_10711_gb300 import build, ucn as U
    build.build()
    return U


def test_library_exports_every_declared_entry_point(ucn):
    names = declared_functions()
    assert "ucn_scp_solve" in names and "ucn_problem_create" in names and len(names) >= 10
    lib = ucn.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_header_structs_match_binding():
    from paper_2603_10711_gb300 import ucn as U
    assert U.STATS_DTYPE.itemsize == 128
    text = open(os.path.join(ROOT, "include", "ucn.h")).read()
    body = text[text.index("typedef struct {\n  int model, nx, nu, batch;"):text.index("} ucn_problem_desc;")]
    # every field of the descriptor appears in the ctypes mirror, in order
    fields = re.findall(r"\b(\w+)\s*(?=[,;])", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    mirror = [f[0] for f in U.ProblemDesc._fields_]
    assert fields == mirror


def create(ucn, prob, **over):
    desc, keep = ucn.make_desc(prob, **over)
    return desc, keep


@pytest.mark.parametrize("mutate,needle", [
    (lambda d: setattr(d, "model", 9), "unknown model"),
    (lambda d: setattr(d, "nx", 5), "needs nx"),
    (lambda d: setattr(d, "batch", 0), "batch"),
    (lambda d: setattr(d, "precision", 7), "precision"),
    (lambda d: setattr(d, "vc_weight", 1.0), "virtual control"),
    (lambda d: setattr(d, "rho_dyn", 0.0), "penalties"),
    (lambda d: setattr(d, "admm_iters", 0), "iteration"),
    (lambda d: setattr(d, "tr_min", -1.0), "trust"),
    (lambda d: setattr(d, "max_obs", 99), "max_obs"),
    (lambda d: setattr(d, "group", 1025), "group must be"),
    (lambda d: setattr(d, "group", -1), "group must be"),
    (lambda d: setattr(d, "group", 3), "not a multiple of group"),
])
def test_create_rejects_bad_descriptors(ucn, mutate, needle):
    prob = W.quad_path(1, seed=0)
    desc, keep = create(ucn, prob)
    mutate(desc)
    h = C.c_void_p()
    rc = ucn.lib().ucn_problem_create(C.byref(desc), C.byref(h))
    assert rc == ucn.UCN_EINVAL
    assert needle in ucn.ucn_last_error()
    assert not h.value


def test_scenario_groups_need_the_quadrotor_model(ucn):
    prob = W.mars_batch(4, seed=1, N=10)
    desc, keep = create(ucn, prob, group=2)
    h = C.c_void_p()
    assert ucn.lib().ucn_problem_create(C.byref(desc), C.byref(h)) == ucn.UCN_EINVAL
    assert "quadrotor" in ucn.ucn_last_error()
    assert ucn.lib().ucn_scp_solve_noalloc(C.byref(desc), None, None, None, None, None, None, None) == ucn.UCN_EINVAL


def test_create_rejects_bad_horizons(ucn):
    prob = W.quad_path(2, seed=0)
    for bad in (0, 256):
        prob.N[1] = bad
        desc, keep = create(ucn, prob)
        h = C.c_void_p()
        assert ucn.lib().ucn_problem_create(C.byref(desc), C.byref(h)) == ucn.UCN_EINVAL
        assert "horizon[1]" in ucn.ucn_last_error()


def test_null_arguments_are_rejected(ucn):
    lib = ucn.lib()
    assert lib.ucn_problem_create(None, None) == ucn.UCN_EINVAL
    assert lib.ucn_scp_solve(None, None, None, None, None, None, None, None) == ucn.UCN_EINVAL
    assert lib.ucn_linearize(None, None, None, None, None, None, None) == ucn.UCN_EINVAL
    assert lib.ucn_state_export(None, None, None) == ucn.UCN_EINVAL
    assert lib.ucn_total_x(None) == -1
    assert lib.ucn_problem_last_launches(None) == -1


def test_double_float_check_validates_before_any_launch(ucn):
    # argument errors return before the library touches a device
    lib = ucn.lib()
    fake = C.c_void_p(16)   # never dereferenced on these paths
    assert lib.ucn_df_check(ucn.UCN_DF_ADD, None, None, None, 0.0, 4, fake, None) == ucn.UCN_EINVAL
    assert lib.ucn_df_check(ucn.UCN_DF_ADD, fake, fake, None, 0.0, -1, fake, None) == ucn.UCN_EINVAL
    assert lib.ucn_df_check(ucn.UCN_DF_ADD, fake, fake, None, 0.0, 4, None, None) == ucn.UCN_EINVAL
    assert lib.ucn_df_check(ucn.UCN_DF_ADD, fake, fake, None, 0.0, 0, fake, None) == ucn.UCN_OK   # nothing to do
    assert lib.ucn_df_check(9, fake, fake, None, 0.0, 4, fake, None) == ucn.UCN_EINVAL          # unknown op
    assert lib.ucn_df_check(ucn.UCN_DF_SQDIFF_SUM, fake, None, None, 0.0, 4, fake, None) == ucn.UCN_EINVAL
    assert lib.ucn_df_check(ucn.UCN_DF_RK4 + 9, fake, fake, fake, 0.1, 4, fake, None) == ucn.UCN_EINVAL
