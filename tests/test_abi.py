"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(CPU only: no compute call needs a GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_06872_gb300 import binding
    return binding.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(gt_[a-z_0-9]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(built):
    names = _declared()
    assert "gt_transpose" in names and "gt_plan_create" in names
    for name in sorted(names):
        assert hasattr(built, name), f"{name} declared in include/ but not exported"


def test_binding_export_list_matches_header(built):
    from paper_2501_06872_gb300 import binding
    assert set(binding.EXPORTS) >= _declared() - {"gt_transpose_batched"}


def test_status_strings_and_version(built):
    built.gt_status_string.restype = ctypes.c_char_p
    assert built.gt_status_string(0) == b"ok"
    assert b"range" in built.gt_status_string(2)
    assert built.gt_version() >= 100


def test_default_config_follows_eq1_sizing(built):
    from paper_2501_06872_gb300 import binding
    c = binding.default_config(1 << 24, 16 << 24)
    assert c.hdv_k > 0 and (1 << c.table_log2) >= 2 * c.hdv_k
    assert c.block_threads % 32 == 0 and c.sample_permille == 10
    small = binding.default_config(1000, 5000)
    assert small.hdv_k == 0  # tiny graphs: pure atomic (Algorithm 1)


def test_plan_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2501_06872_gb300 import binding
    with pytest.raises(binding.GtError) as ei:
        binding.Plan(100, 1000, False)
    assert ei.value.code in (5,)  # GT_ERR_CUDA


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2501_06872_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.load()
