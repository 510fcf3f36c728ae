"""C-ABI checks that need no GPU: the library builds and loads, exports every
function that include/rde_chem.h and include/rde_chem_selftest.h declare, and rejects malformed or inconsistent
mechanism text on the host before touching the device."""
import ctypes as C
import os
import re

import pytest

from paper_2508_16105_gb300 import build, rde_chem, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return rde_chem.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rde_chem.h")).read()
    src += open(os.path.join(ROOT, "include", "rde_chem_selftest.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rde_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def load_err(text):
    h = C.c_void_p()
    b = text.encode()
    rc = rde_chem.load_library().rde_mech_load(b, len(b), 0, C.byref(h))
    return rc, rde_chem.load_library().rde_last_error_message().decode()


def test_parse_errors(lib):
    good = synth.h2_air_mechanism().to_text()
    assert load_err("hello")[0] == -3
    assert load_err(good.replace("RDEMECH 1", "RDEMECH 2"))[0] == -3
    assert load_err(good.replace("\nEND\n", "\n"))[0] == -3
    rc, msg = load_err(good.replace("RX ELEM REV", "RX BOGUS REV", 1))
    assert rc == -3 and "unknown reaction type" in msg


def test_validation_errors(lib):
    good = synth.h2_air_mechanism().to_text()
    # element imbalance: H + O2 <=> O + OH becomes H + O2 <=> O + H2O
    bad = good.replace("2 H 1 O2 1 2 O 1 OH 1", "2 H 1 O2 1 2 O 1 H2O 1", 1)
    assert bad != good
    rc, msg = load_err(bad)
    assert rc == -4 and "not balanced" in msg
    m = synth.isomer_mechanism()
    t = m.to_text().replace("SP A 20", "SP A -20")
    assert load_err(t)[0] == -4
    t = m.to_text().replace("1 A 1 1 B 1", "1 Q 1 1 B 1")
    rc, msg = load_err(t)
    assert rc == -4 and "unknown species" in msg
    lind = synth.isomer_mechanism(kind="LINDEMANN", low=(1e12, 0, 0)).to_text()
    rc, msg = load_err("\n".join(l for l in lind.splitlines() if not l.startswith("LOW")) + "\n")
    assert rc == -4 and "LOW" in msg


def test_null_and_args(lib):
    assert lib.rde_mech_load(None, 0, 0, None) == -1
    assert lib.rde_mech_free(None) == 0
    assert lib.rde_chem_advance(None, 0, None, None, None, 1.0, None) == -1
    o = rde_chem.rde_chem_options()
    assert lib.rde_chem_default_options(C.byref(o)) == 0
    assert (o.rtol, o.atol, o.max_substeps) == (1e-8, 1e-12, 100000)
    assert lib.rde_strerror(-3).decode() == "mechanism text malformed"
