"""The C-ABI library builds, loads and exports every declared symbol; host
argument checks reject bad calls before any device work (no GPU needed)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2110_02820_gb300 import build, nyspcg
    build.build()
    return nyspcg.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["nys_sketch", "nys_sketch_adaptive", "nys_precond_apply", "pcg_solve",
                     "nys_factor_get", "nys_factor_free", "nys_status_str", "nys_op_matvec",
                     "nys_power_err_est"]:
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings(L):
    from paper_2110_02820_gb300 import nyspcg as ny
    assert ny.status_str(0) == "ok"
    assert "argument" in ny.status_str(1)
    assert ny.status_str(99) == "unknown status"


def _op(kind=0, dtype=0, n=64, m=0, d=0, ld=64, data=0x1000, sigma=0.0):
    from paper_2110_02820_gb300.nyspcg import _Operator
    return _Operator(kind, dtype, n, m, d, ld, data, sigma)


def test_host_argument_checks_reject_before_device_work(L):
    from paper_2110_02820_gb300 import nyspcg as ny
    h = C.c_void_p()
    # null operator / null output
    assert L.nys_sketch(None, 4, 0, None, 0, C.byref(h), None) == ny.NYS_ERR_ARG
    op = _op()
    assert L.nys_sketch(C.byref(op), 4, 0, None, 0, None, None) == ny.NYS_ERR_ARG
    # ell > n, ell < 1, bad precision
    assert L.nys_sketch(C.byref(op), 65, 0, None, 0, C.byref(h), None) == ny.NYS_ERR_ARG
    assert L.nys_sketch(C.byref(op), 0, 0, None, 0, C.byref(h), None) == ny.NYS_ERR_ARG
    assert L.nys_sketch(C.byref(op), 4, 0, None, 7, C.byref(h), None) == ny.NYS_ERR_ARG
    # dense operator must be FP64, ld >= n, data 16-byte aligned
    assert L.nys_sketch(C.byref(_op(dtype=1)), 4, 0, None, 0, C.byref(h), None) == ny.NYS_ERR_ARG
    assert L.nys_sketch(C.byref(_op(ld=10)), 4, 0, None, 0, C.byref(h), None) == ny.NYS_ERR_ARG
    assert L.nys_sketch(C.byref(_op(data=0x1004)), 4, 0, None, 0, C.byref(h), None) == ny.NYS_ERR_ARG
    # RBF: sigma > 0, 1 <= d <= 64
    assert L.nys_sketch(C.byref(_op(kind=2, dtype=1, d=3, ld=3, sigma=0.0)), 4, 0, None, 0,
                        C.byref(h), None) == ny.NYS_ERR_ARG
    assert L.nys_sketch(C.byref(_op(kind=2, dtype=1, d=65, ld=65, sigma=1.0)), 4, 0, None, 0,
                        C.byref(h), None) == ny.NYS_ERR_ARG
    # gram: m > 0
    assert L.nys_sketch(C.byref(_op(kind=1, dtype=1, m=0)), 4, 0, None, 0, C.byref(h),
                        None) == ny.NYS_ERR_ARG


def test_pcg_argument_checks(L):
    from paper_2110_02820_gb300 import nyspcg as ny
    op = _op()
    res = (ny._PcgResult * 2)()
    mu = (C.c_double * 2)(1e-3, -1.0)
    # negative mu
    assert L.pcg_solve(C.byref(op), None, mu, 2, C.c_void_p(0x2000), C.c_void_p(0x3000), None, res,
                       None) == ny.NYS_ERR_ARG
    mu = (C.c_double * 2)(1e-3, 1e-3)
    # null b / x / results, nsys < 1
    assert L.pcg_solve(C.byref(op), None, mu, 2, None, C.c_void_p(0x3000), None, res, None) == ny.NYS_ERR_ARG
    assert L.pcg_solve(C.byref(op), None, mu, 0, C.c_void_p(0x2000), C.c_void_p(0x3000), None, res,
                       None) == ny.NYS_ERR_ARG
    # bad options: mixed with inner_tol outside (0, 1)
    opts = ny._PcgOpts(1e-8, 100, ny.NYS_PREC_MIXED, 2.0, 5, 0, None)
    assert L.pcg_solve(C.byref(op), None, mu, 2, C.c_void_p(0x2000), C.c_void_p(0x3000),
                       C.byref(opts), res, None) == ny.NYS_ERR_ARG
    # adaptive: ratio rule needs mu > 0; err rule needs q >= 1
    h = C.c_void_p()
    assert L.nys_sketch_adaptive(C.byref(op), 4, 16, ny.NYS_RULE_RATIO, 10.0, 0, 0.0, 0, None, None,
                                 0, C.byref(h), None, None) == ny.NYS_ERR_ARG
    assert L.nys_sketch_adaptive(C.byref(op), 4, 16, ny.NYS_RULE_ERR, 1.0, 0, 1.0, 0, None, None,
                                 0, C.byref(h), None, None) == ny.NYS_ERR_ARG
    assert L.nys_sketch_adaptive(C.byref(op), 4, 65, ny.NYS_RULE_ERR, 1.0, 5, 1.0, 0, None, None,
                                 0, C.byref(h), None, None) == ny.NYS_ERR_ARG
    # precond apply: null factor
    assert L.nys_precond_apply(None, mu, 1, C.c_void_p(0x2000), C.c_void_p(0x3000), 0,
                               None) == ny.NYS_ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2110_02820_gb300 import nyspcg as ny
    monkeypatch.setattr(ny, "_lib", None)
    monkeypatch.setattr(ny, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ny.NysLibraryMissing):
        ny.lib()


def test_newer_entry_points_reject_bad_arguments(L):
    # column sketch, block PCG, regularization path and sketch-and-solve check
    # their arguments on the host and return NYS_ERR_ARG before any device work
    from paper_2110_02820_gb300 import nyspcg as ny
    i64, dbl, vp, u64, i32 = C.c_int64, C.c_double, C.c_void_p, C.c_uint64, C.c_int32
    op = _op()
    h = C.c_void_p()
    cols = L.nys_sketch_columns
    assert cols(C.byref(op), i64(4), u64(0), None, i32(0), None, None) == ny.NYS_ERR_ARG
    assert cols(C.byref(op), i64(65), u64(0), None, i32(0), C.byref(h), None) == ny.NYS_ERR_ARG
    assert cols(C.byref(op), i64(0), u64(0), None, i32(0), C.byref(h), None) == ny.NYS_ERR_ARG
    assert cols(C.byref(op), i64(4), u64(0), None, i32(7), C.byref(h), None) == ny.NYS_ERR_ARG

    res = (ny._PcgResult * 40)()
    b, x = vp(0x2000), vp(0x3000)
    blk = L.nys_block_pcg
    for nrhs, mu in ((0, 1e-3), (33, 1e-3), (4, -1.0), (4, float("nan"))):
        assert blk(C.byref(op), None, dbl(mu), i64(nrhs), b, x, None, res, None) == ny.NYS_ERR_ARG
    assert blk(C.byref(op), None, dbl(1e-3), i64(4), None, x, None, res, None) == ny.NYS_ERR_ARG

    pres = (ny._PathResult * 4)()
    path = L.nys_reg_path
    good = (C.c_double * 3)(1e-1, 1e-2, 1e-3)
    bad = (C.c_double * 3)(1e-1, 0.0, 1e-3)

    def call(count=3, mus=good, ell0=4, ell_max=16, err_factor=30.0, q=5):
        return path(C.byref(op), i64(count), mus, b, x, i64(ell0), i64(ell_max), dbl(err_factor),
                    i32(q), u64(0), None, None, None, pres, None)
    assert call(count=0) == ny.NYS_ERR_ARG
    assert call(mus=bad) == ny.NYS_ERR_ARG
    assert call(ell0=32, ell_max=16) == ny.NYS_ERR_ARG
    assert call(ell_max=65) == ny.NYS_ERR_ARG
    assert call(err_factor=0.0) == ny.NYS_ERR_ARG
    assert call(q=0) == ny.NYS_ERR_ARG

    mu1 = (C.c_double * 1)(1e-3)
    assert L.nys_sketch_solve(None, mu1, i64(1), b, x, i32(0), None) == ny.NYS_ERR_ARG


def test_generator_krr_and_probe_entry_points_reject_bad_arguments(L):
    # Philox, the random stream, the KRR objective / gradients and the unit
    # probe check their arguments on the host before any device work
    from paper_2110_02820_gb300 import nyspcg as ny
    i64, dbl, vp, u64, i32 = C.c_int64, C.c_double, C.c_void_p, C.c_uint64, C.c_int32
    L.nys_philox4x32_10.argtypes = [vp, vp, i64, vp, vp]
    L.nys_philox4x32_10.restype = i32
    assert L.nys_philox4x32_10(None, vp(0x1000), 4, vp(0x2000), None) == ny.NYS_ERR_ARG
    assert L.nys_philox4x32_10(vp(0x1000), vp(0x1000), -1, vp(0x2000), None) == ny.NYS_ERR_ARG
    L.nys_random_stream.argtypes = [u64, u64, i64, i64, vp, vp, vp]
    L.nys_random_stream.restype = i32
    assert L.nys_random_stream(1, 2, -1, 4, vp(0x1000), None, None) == ny.NYS_ERR_ARG
    assert L.nys_random_stream(1, 2, 0, -4, vp(0x1000), None, None) == ny.NYS_ERR_ARG
    assert L.nys_random_stream(1, 2, 0, 4, None, None, None) == ny.NYS_ERR_ARG

    L.nys_krr_validation.argtypes = [vp, i64, i64, vp, i64, i64, i64, dbl, vp, vp,
                                     C.POINTER(dbl), vp, vp, vp]
    L.nys_krr_validation.restype = i32
    loss = dbl()
    P, V, a, y, g, k = (vp(0x1000 * (i + 1)) for i in range(6))
    # d out of range, sigma <= 0, aliasing outputs
    assert L.nys_krr_validation(P, 10, 70, V, 5, 70, 65, 1.0, a, y, C.byref(loss), g, k,
                                None) == ny.NYS_ERR_ARG
    assert L.nys_krr_validation(P, 10, 4, V, 5, 4, 4, 0.0, a, y, C.byref(loss), g, k,
                                None) == ny.NYS_ERR_ARG
    assert L.nys_krr_validation(P, 10, 4, V, 5, 4, 4, 1.0, a, y, C.byref(loss), g, g,
                                None) == ny.NYS_ERR_ARG
    L.nys_krr_gradients.argtypes = [vp, i64, i64, vp, i64, i64, i64, dbl, vp, vp, vp,
                                    C.POINTER(dbl), vp]
    L.nys_krr_gradients.restype = i32
    out = (dbl * 2)()
    assert L.nys_krr_gradients(P, 10, 4, None, 0, 0, 4, 1.0, None, a, None, out,
                               None) == ny.NYS_ERR_ARG
    assert L.nys_krr_gradients(P, 10, 4, V, 5, 4, 4, 1.0, a, a, None, out,
                               None) == ny.NYS_ERR_ARG  # validation points need g
    L.nys_unit_peak.argtypes = [i32, C.POINTER(dbl), vp]
    L.nys_unit_peak.restype = i32
    r = dbl()
    assert L.nys_unit_peak(3, C.byref(r), None) == ny.NYS_ERR_ARG
    assert L.nys_unit_peak(0, None, None) == ny.NYS_ERR_ARG
