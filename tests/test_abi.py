"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no GPU needed; no compute calls)."""
import glob
import os
import re

from paper_2502_18929_gb300 import qmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for path in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(path).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(qmc_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("qmc_create", "qmc_load_schedule", "qmc_init_populations", "qmc_step", "qmc_observables",
              "qmc_export", "qmc_checkpoint", "qmc_restore", "qmc_destroy", "qmc_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = qmc.lib()
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header():
    assert set(qmc.EXPORTED) <= declared_functions()


def test_create_fails_loudly_without_a_device():
    import torch
    if torch.cuda.is_available():
        return
    try:
        qmc.QMC(4, 2, 1, 100)
    except qmc.QmcError as e:
        assert e.code in (qmc.ERR_CUDA, qmc.ERR_OOM)
    else:
        raise AssertionError("context creation must fail without a CUDA device")


def test_invalid_config_rejected():
    import ctypes as C
    L = qmc.lib()
    h = C.c_void_p()
    cfg = qmc.Config(61, 1, 1, 0, 1, 100, 0, 0, 0, None)   # 61 qubits: beyond the 60 supported
    assert L.qmc_create(C.byref(h), C.byref(cfg)) == qmc.ERR_INVALID_ARG
    cfg = qmc.Config(8, 1, 1, 0, 1, 100, 0, 0, 0, None)
    cfg.alloc = qmc.ALLOC_FN(lambda b, s, u: None)         # an allocator without its free
    assert L.qmc_create(C.byref(h), C.byref(cfg)) in (qmc.ERR_INVALID_ARG, qmc.ERR_CUDA)
