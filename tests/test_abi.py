"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/mcgb.h declares; without a GPU it refuses to create a context
(no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "mcgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcgb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libmcgb():
    import paper_2501_05440_gb300 as m
    path = m.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = declared_entry_points()
    for required in ["mcgb_create", "mcgb_run_eigenvalue", "mcgb_run_fixed_source", "mcgb_get_tally",
                     "mcgb_get_k", "mcgb_backward_fixed", "mcgb_batch_run", "mcgb_batch_autotune"]:
        assert required in names
    assert len(names) >= 38


def test_library_exports_every_declared_symbol(libmcgb):
    missing = [n for n in declared_entry_points() if not hasattr(libmcgb, n)]
    assert not missing, missing


def test_create_without_gpu_fails_loudly(libmcgb):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2501_05440_gb300 as m
    with pytest.raises(m.McgbError) as e:
        m.Context()
    assert e.value.code == -3


def test_binding_names_match_the_c_calls():
    import paper_2501_05440_gb300 as m
    for n in declared_entry_points():
        short = n[len("mcgb_"):]
        if short in ("create", "destroy", "last_error"):
            continue
        if short.endswith("_noalloc"):
            assert hasattr(m, short), n
            continue
        if short.startswith("batch_"):
            attr = short[len("batch_"):]
            if attr in ("create", "destroy"):
                continue
            assert hasattr(m.Batch, {"add_problem": "add_problem", "tally": "tally",
                                     "counters": "counters"}.get(attr, attr)), n
        else:
            assert hasattr(m.Context, short), n
