"""Host-side checks of the C ABI (no GPU): the library builds, loads and
exports every entry point include/ptebd.h declares, and the pure host logic
(config validation, buffer sizing) answers as documented."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptebd.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(ptebd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2312_02667_gb300 import build
    if not os.path.exists(build.LIB):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("no nvcc to build libptebd")
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ptebd_create", "ptebd_apply_layer", "ptebd_apply_bonds", "ptebd_regauge", "ptebd_norm",
                 "ptebd_overlap", "ptebd_expect", "ptebd_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2312_02667_gb300 import ptebd
    assert sorted(set(ptebd.EXPORTS) | {"ptebd_last_error"}) == declared_symbols()
    for s in declared_symbols():
        if s != "ptebd_last_error":
            assert hasattr(ptebd, s), s


def test_required_bytes_and_validation(lib_path):
    from paper_2312_02667_gb300 import ptebd
    cfg = ptebd.make_config(1024, 256, "mixed", 1e-12, 1)
    sb, wb, wmin = ptebd.ptebd_required_bytes(cfg)
    # Gamma store: 1024 sites x 2 x 256 x 256 complex64 = 1 GiB
    assert sb >= 1024 * 2 * 256 * 256 * 8
    # whole-layer workspace: 512 slots of two 512x512 complex64 matrices
    assert wb >= 512 * 2 * 512 * 512 * 8
    assert wmin < wb and wmin >= 2 * 512 * 512 * 8
    # the FP64 resolution adds two 512x512 complex128 matrices per slot
    assert wb >= 512 * (3 * 512 * 512 * 8 + 2 * 512 * 512 * 16)
    plain = ptebd.make_config(1024, 256, "mixed", 1e-12, 1, resolve=0.0)
    sbp, wbp, _ = ptebd.ptebd_required_bytes(plain)
    assert sbp == sb and wbp <= wb - 512 * 2 * 512 * 512 * 16
    cfg64 = ptebd.make_config(1024, 256, "fp64")
    sb64, wb64, _ = ptebd.ptebd_required_bytes(cfg64)
    assert sb64 > 1.9 * sb and wb64 > 1.9 * wbp
    bad = ptebd.make_config(16, 8)
    bad.d = 3
    with pytest.raises(ptebd.PtebdError) as e:
        ptebd.ptebd_required_bytes(bad)
    assert e.value.code == -2
    for field, value in (("n_sites", 1), ("chi_max", 0), ("chi_max", 4096), ("precision", 7), ("g", -1)):
        c = ptebd.make_config(16, 8)
        setattr(c, field, value)
        with pytest.raises(ptebd.PtebdError):
            ptebd.ptebd_required_bytes(c)
    c = ptebd.make_config(16, 8, cutoff=-1.0)
    with pytest.raises(ptebd.PtebdError):
        ptebd.ptebd_required_bytes(c)


def test_create_rejects_bad_buffers_without_touching_the_device(lib_path):
    from paper_2312_02667_gb300 import ptebd
    cfg = ptebd.make_config(16, 8)
    sb, wb, _ = ptebd.ptebd_required_bytes(cfg)
    with pytest.raises(ptebd.PtebdError) as e:
        ptebd.ptebd_create(cfg, 0, sb, 0, wb, 0)
    assert e.value.code == -1
    with pytest.raises(ptebd.PtebdError) as e:
        ptebd.ptebd_create(cfg, 0x1001, sb, 0x2000, wb, 0)  # misaligned
    assert e.value.code == -3
    with pytest.raises(ptebd.PtebdError) as e:
        ptebd.ptebd_create(cfg, 0x1000, sb - 1, 0x2000, wb, 0)  # too small
    assert e.value.code == -3
