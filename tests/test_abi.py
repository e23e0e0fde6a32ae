"""C ABI checks that need no GPU: the library builds, loads, and exports
exactly the entry points include/twed.h declares."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "twed.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(twed_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2007_16135_gb300 import build
    return build.build()


def test_header_and_binding_agree():
    from paper_2007_16135_gb300 import twed
    assert declared_functions() == sorted(twed.EXPORTS)


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (twed_[a-z0-9_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_reports_version(lib_path):
    from paper_2007_16135_gb300 import twed
    lib = twed.load(lib_path)
    for name in twed.EXPORTS:
        assert hasattr(lib, name)
    assert twed.version().startswith("twed-gb300")


def test_no_gpu_means_loud_failure(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2007_16135_gb300 import twed
    with pytest.raises(twed.TwedError):
        twed.Handle()


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "use.c"
    src.write_text('#include "twed.h"\nint main(void){twed_handle_t h=0;(void)h;return 0;}\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-c", str(src), "-o", str(tmp_path / "use.o")], check=True)


def test_kernels_use_no_oracle_code():
    # the CUDA path and the oracle share nothing: no include, import or path
    csrc = os.path.join(ROOT, "paper_2007_16135_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|twed_oracle|liboracle",
                                     text, flags=re.M), f
