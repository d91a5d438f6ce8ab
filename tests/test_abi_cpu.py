"""The C ABI library loads and exports every symbol the headers in include/
declare (no GPU needed: only dlopen/dlsym, no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


HEADERS = ("muca.h", "muca_probe.h")


def declared_symbols():
    assert sorted(HEADERS) == sorted(f for f in os.listdir(os.path.join(ROOT, "include"))
                                     if f.endswith(".h"))
    names = set()
    for h in HEADERS:
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(muca_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("muca_init", "muca_sweep_iter", "muca_merge_update", "muca_reweight",
              "muca_run_graph", "muca_destroy", "muca_set_window", "muca_probe_int",
              "muca_probe_l2_read"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1502_07214_gb300 import build, muca

    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing
    # the binding's table covers the header
    assert set(declared_symbols()) <= set(muca.SIGNATURES)


def test_binding_raises_without_gpu_instead_of_falling_back():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1502_07214_gb300 import muca

    with pytest.raises(muca.MucaError) as e:
        muca.Context([{"L": 4, "T": 1.0, "n_walkers": 4}], stream=0)
    # the failure is a CUDA error reported through the status code and the
    # last-error text, not a silent CPU run
    assert e.value.code in (muca.ERR_CUDA, muca.ERR_OOM)
    assert muca.last_error()


def test_invalid_arguments_are_rejected_before_any_device_work():
    from paper_1502_07214_gb300 import muca

    with pytest.raises(muca.MucaError) as e:
        muca.Context([{"L": 1, "T": 1.0, "n_walkers": 4}], stream=0)
    assert e.value.code == muca.ERR_INVALID_ARG
    with pytest.raises(muca.MucaError) as e:
        muca.Context([{"L": 4, "T": -1.0, "n_walkers": 4}], stream=0)
    assert e.value.code == muca.ERR_INVALID_ARG
    with pytest.raises(muca.MucaError) as e:
        muca.Context([{"L": 4, "T": 1.0, "n_walkers": 4, "e_min": 10, "e_max": 5}], stream=0)
    assert e.value.code == muca.ERR_INVALID_ARG


def test_binding_constants_match_the_header():
    """Every value the header defines (status codes, residencies, recursions,
    limits) has the same value in the binding."""
    from paper_1502_07214_gb300 import muca

    text = open(os.path.join(ROOT, "include", "muca.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define MUCA_([A-Z_0-9]+)\s+\(?(-?\d+)\)?", text)}
    assert {"OK", "ERR_INVALID_ARG", "RES_SPLIT", "REC_ACCUMULATED", "MAX_L", "NK"} <= set(defs)
    for name, value in defs.items():
        assert getattr(muca, name) == value, name
