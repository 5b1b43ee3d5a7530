"""The C-ABI library: it builds for sm_103a and exports every symbol of include/gbc.h.
CPU only (no compute call is made without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gbc_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_builds_and_exports_header_symbols():
    import paper_2403_07858_gb300 as gbc
    path = gbc.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gbc_[a-z0-9_]+)", out))
    declared = _declared_functions()
    assert declared, "no declarations found"
    assert declared <= exported, sorted(declared - exported)
    # the Python binding knows every declared entry point
    assert declared <= set(gbc.SIGNATURES), sorted(declared - set(gbc.SIGNATURES))


def test_library_loads_and_fails_loudly_without_gpu():
    import paper_2403_07858_gb300 as gbc
    lib = gbc.load_library()
    for name in _declared_functions():
        assert hasattr(lib, name)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        with pytest.raises(gbc.GbcError):
            gbc.Context(0)


def test_oracle_is_not_linked_into_the_product():
    import paper_2403_07858_gb300 as gbc
    out = subprocess.run(["nm", "-D", gbc.build()], capture_output=True, text=True, check=True).stdout
    assert "orc_" not in out
    src = open(os.path.join(ROOT, "paper_2403_07858_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_traffic_record_tracks_kernel_code_not_comments(tmp_path, monkeypatch):
    """bench.py reports the committed DRAM traffic of the enumeration kernel
    only while the kernel source (comments and whitespace aside) is the one
    the counters were taken on."""
    import importlib.util
    import json
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    src = os.path.join(root, "paper_2403_07858_gb300", "csrc", "gbc_search.cu")
    text = open(src).read()
    fake = tmp_path / "repo"
    (fake / "paper_2403_07858_gb300" / "csrc").mkdir(parents=True)
    (fake / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(fake))

    def digest_of(t):
        (fake / "paper_2403_07858_gb300" / "csrc" / "gbc_search.cu").write_text(t)
        return bench.kernel_source_digest()

    d0 = digest_of(text)
    assert digest_of("// a new comment\n" + text.replace("\n", "\n  ", 3)) == d0
    assert digest_of(text + "\nint extra_code;\n") != d0
    json.dump({"source_digest": d0, "dram_bytes_per_launch_scaled": 123.0}, open(fake / "profiles" / "enumerate_traffic.json", "w"))
    digest_of(text)
    assert bench._ncu_traffic() == 123.0
    digest_of(text + "\nint extra_code;\n")
    assert bench._ncu_traffic() is None
