"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/gbresample.h declares (no compute call: no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbresample.h")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_A-Z0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_01356_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ["rs_create", "rs_destroy", "rs_resample_w", "rs_resample_W", "rs_sorted_uniform", "rs_cumulative",
                 "rs_map", "rs_philox", "rs_resample_batched", "rs_get_status", "rs_last_error", "rs_version"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_version(libpath):
    import paper_2604_01356_gb300 as g
    L = g.lib()
    for n in declared():
        assert hasattr(L, n)
    assert g.rs_version().startswith("gbresample")


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "gbresample.h"\nint main(void){rs_opts o={0}; (void)o; return (int)RS_OK;}\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                    "-o", str(tmp_path / "t.o")], check=True)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2604_01356_gb300._binding as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b, "library_path", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        b.lib()


def test_oracle_and_library_share_no_code():
    """The oracle is independent of the CUDA path: no includes or imports across."""
    orc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "gbresample" not in orc and "csrc" not in orc
    pkg = os.path.join(ROOT, "paper_2604_01356_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "oracle.c" not in txt, f
