"""C ABI checks that need no GPU: exported symbols, status strings, and the
host-side validation and planning behind every entry point."""
import ctypes
import re
from pathlib import Path

import pytest
import torch

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    src = (ROOT / "include" / "cbp.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:cbp_status|const char\*|size_t)\s+(cbp_\w+)\s*\(", src, re.M)))


def test_every_declared_symbol_is_exported(built_lib):
    from paper_1203_4874_gb300 import cbp
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(built_lib, n), n
    assert sorted(cbp.EXPORTED) == names


def test_status_strings(built_lib):
    from paper_1203_4874_gb300 import cbp
    assert cbp.status_string(0) == "CBP_OK"
    assert cbp.status_string(-3) == "CBP_ERR_NOT_COPRIME"
    assert cbp.status_string(12345) == "CBP_UNKNOWN_STATUS"


def _frames(n, c, h, w, dtype=0, rs=0):
    from paper_1203_4874_gb300 import cbp
    return cbp.cbp_frames(0x1000, n, c, h, w, dtype, rs, 0, 0)


def _ws(b1, b2, prm):
    from paper_1203_4874_gb300 import cbp
    out = ctypes.c_size_t()
    s = cbp.lib().cbp_workspace_size(ctypes.byref(b1), ctypes.byref(b2), ctypes.byref(prm),
                                     ctypes.byref(out))
    return s, out.value


def test_planner_accepts_the_workload_shapes(built_lib):
    from paper_1203_4874_gb300 import cbp
    for (h, w, c, t1, t2, path, n) in [(64, 64, 1, 5, 5, "fp64", 1), (480, 640, 1, 9, 11, "fp64", 30),
                                       (1080, 1920, 3, 15, 17, "mixed", 60)]:
        s, b = _ws(_frames(n, c, h + t1 - 1, w + t1 - 1), _frames(n, c, h + t2 - 1, w + t2 - 1),
                   cbp.params(t1, t2, path=path))
        assert s == cbp.CBP_OK and b > 0


def test_planner_rejects_bad_arguments(built_lib):
    from paper_1203_4874_gb300 import cbp
    ok1, ok2 = _frames(1, 1, 68, 68), _frames(1, 1, 68, 68)
    assert _ws(ok1, ok2, cbp.params(5, 5))[0] == cbp.CBP_OK
    # blurred sizes inconsistent with t1 - t2
    assert _ws(ok1, _frames(1, 1, 70, 68), cbp.params(5, 7))[0] == cbp.CBP_ERR_SIZE_MISMATCH
    # fewer samples than the kernel height
    assert _ws(ok1, ok2, cbp.params(5, 5, m=4))[0] == cbp.CBP_ERR_INVALID_ARG
    # library limits
    assert _ws(ok1, ok2, cbp.params(5, 5, m=33))[0] == cbp.CBP_ERR_UNSUPPORTED
    assert _ws(_frames(1, 1, 200, 200), _frames(1, 1, 200, 200),
               cbp.params(40, 40))[0] == cbp.CBP_ERR_UNSUPPORTED
    # FFT grid must hold the frames and be 7-smooth
    assert _ws(ok1, ok2, cbp.params(5, 5, pad_h=66))[0] == cbp.CBP_ERR_INVALID_ARG
    assert _ws(ok1, ok2, cbp.params(5, 5, pad_h=88))[0] == cbp.CBP_ERR_INVALID_ARG   # 88 = 8 * 11
    assert _ws(ok1, ok2, cbp.params(5, 5, pad_h=72, pad_w=75))[0] == cbp.CBP_OK
    # negative eps, mismatched batch / dtype, bad strides, null data
    assert _ws(ok1, ok2, cbp.params(5, 5, eps=-1.0))[0] == cbp.CBP_ERR_INVALID_ARG
    assert _ws(ok1, _frames(2, 1, 68, 68), cbp.params(5, 5))[0] == cbp.CBP_ERR_INVALID_ARG
    assert _ws(ok1, _frames(1, 1, 68, 68, dtype=1), cbp.params(5, 5))[0] == cbp.CBP_ERR_INVALID_ARG
    assert _ws(_frames(1, 1, 68, 68, rs=10), ok2, cbp.params(5, 5))[0] == cbp.CBP_ERR_INVALID_ARG
    null = cbp.cbp_frames(0, 1, 1, 68, 68, 0, 0, 0, 0)
    assert _ws(null, ok2, cbp.params(5, 5))[0] == cbp.CBP_ERR_INVALID_ARG
    # no latent left
    assert _ws(_frames(1, 1, 4, 4), _frames(1, 1, 4, 4), cbp.params(5, 5))[0] == cbp.CBP_ERR_SIZE_MISMATCH


def test_workspace_grows_with_batch(built_lib):
    from paper_1203_4874_gb300 import cbp
    prm = cbp.params(9, 11)
    _, one = _ws(_frames(1, 1, 488, 648), _frames(1, 1, 490, 650), prm)
    _, ten = _ws(_frames(10, 1, 488, 648), _frames(10, 1, 490, 650), prm)
    assert 9 * one < ten < 11 * one


def test_create_fails_cleanly_without_device(built_lib):
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1203_4874_gb300 import cbp
    ctx = ctypes.c_void_p()
    assert cbp.lib().cbp_create(ctypes.byref(ctx), 0, 0) == cbp.CBP_ERR_CUDA
    assert cbp.lib().cbp_create(None, 0, 0) == cbp.CBP_ERR_INVALID_ARG


@pytest.mark.skipif(torch.cuda.is_available(), reason="an accepted call would launch kernels on "
                    "the placeholder addresses; the size check is pinned where no GPU is present")
def test_noalloc_size_check_on_the_1080p_rgb_workload(built_lib):
    """The allocation-free entry point's fixed 16 MiB array holds one 1080p RGB
    pair (15x15 and 17x17 kernels) on either path -- the call gets past the size
    check and fails only for want of a device -- and refuses three pairs."""
    from paper_1203_4874_gb300 import cbp
    for path in ("fp64", "mixed"):
        for n, accepted in ((1, True), (3, False)):
            b1 = _frames(n, 3, 1094, 1934)
            b2 = _frames(n, 3, 1096, 1936)
            prm = cbp.params(15, 17, path=path)
            s = cbp.lib().cbp_estimate_kernels_noalloc(ctypes.byref(b1), ctypes.byref(b2),
                                                       ctypes.byref(prm), ctypes.c_void_p(0x2000),
                                                       ctypes.c_void_p(0x3000), None, None)
            if accepted:
                assert s == cbp.CBP_ERR_CUDA, (path, n, s)
            else:
                assert s == cbp.CBP_ERR_UNSUPPORTED, (path, n, s)


def test_scale_variant_flags_validated(built_lib):
    from paper_1203_4874_gb300 import cbp
    f1, f2 = _frames(1, 1, 68, 68), _frames(1, 1, 68, 68)
    assert _ws(f1, f2, cbp.params(5, 5, m=7, flags=cbp.CBP_FLAG_SCALE_SUPPORT))[0] == cbp.CBP_OK
    assert _ws(f1, f2, cbp.params(5, 5, flags=cbp.CBP_FLAG_SCALE_SUPPORT))[0] == cbp.CBP_ERR_INVALID_ARG
    both = cbp.CBP_FLAG_SCALE_SUPPORT | cbp.CBP_FLAG_K1_ONLY
    assert _ws(f1, f2, cbp.params(5, 5, m=7, flags=both))[0] == cbp.CBP_ERR_INVALID_ARG
    assert _ws(f1, f2, cbp.params(5, 5, flags=cbp.CBP_FLAG_K1_ONLY))[0] == cbp.CBP_OK


def test_size_and_encrypt_validation(built_lib):
    from paper_1203_4874_gb300 import cbp
    import ctypes
    L = cbp.lib()
    t1 = (ctypes.c_int32 * 1)()
    t2 = (ctypes.c_int32 * 1)()
    # blurred sizes that disagree on t1 - t2
    s = L.cbp_estimate_size(ctypes.c_void_p(1), ctypes.byref(_frames(1, 1, 70, 68)),
                            ctypes.byref(_frames(1, 1, 68, 68)), None, t1, t2, None, None, None, None)
    assert s == cbp.CBP_ERR_SIZE_MISMATCH
    prm = cbp.cbp_encrypt_params(0, 5, 0, 0, 0, 0, 0.0, 0.0, 1, 0, 0)
    s = L.cbp_encrypt(ctypes.c_void_p(1), ctypes.c_void_p(0x1000), 1, 1, 8, 8, cbp.CBP_F32, ctypes.byref(prm),
                      ctypes.c_void_p(0x2000), ctypes.c_void_p(0x3000), ctypes.c_void_p(0x4000),
                      ctypes.c_void_p(0x5000), None, None, None, None, None, None)
    assert s == cbp.CBP_ERR_INVALID_ARG
    assert L.cbp_truncate_lsb(ctypes.c_void_p(1), ctypes.c_void_p(0x1000), cbp.CBP_F32, 10, 16, 16,
                              ctypes.c_void_p(0x1000), None) == cbp.CBP_ERR_INVALID_ARG


def test_check_words_need_the_checked_build(built_lib):
    """cbp_check_words and cbp_check_expire_waits answer CBP_ERR_UNSUPPORTED
    in the normal build (no device call); both builds export every declared
    symbol."""
    from paper_1203_4874_gb300 import cbp
    import pytest as _pt
    with _pt.raises(cbp.CbpError) as e:
        cbp.cbp_check_words()
    assert e.value.status == cbp.CBP_ERR_UNSUPPORTED
    with _pt.raises(cbp.CbpError) as e:
        cbp.cbp_check_expire_waits(True)
    assert e.value.status == cbp.CBP_ERR_UNSUPPORTED
    import ctypes
    checked = ctypes.CDLL(str(cbp.LIB_PATH.with_name("libcbp_checks.so")))
    for name in declared_functions():
        assert hasattr(checked, name), name
