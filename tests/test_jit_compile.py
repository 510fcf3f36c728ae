"""The mechanism-specialised kernel source compiles for sm_103a (NVRTC, no GPU needed).

Generation is checked structurally: one descriptor per reaction, the
efficiency terms of third-body reactions written out, the falloff constants
present as exact hexadecimal literals, and ln A / E/R left as run-time reads.
"""
import re

import pytest

from gpu_util import library
from paper_2508_16105_gb300 import rde_chem, synth


def _compile(text, part=0):
    library()
    try:
        return rde_chem.rde_selftest_jit_compile(text, part)
    except rde_chem.RdeError as e:
        if "not found" in str(e) or "lacks an entry point" in str(e):
            pytest.skip("NVRTC is not available: " + str(e))
        raise


def test_h2_mechanism_compiles():
    mech = synth.h2_air_mechanism(16105)
    r = _compile(mech.to_text())
    src = r["source"]
    assert r["cubin_bytes"] > 0
    assert len(re.findall(r"^struct Rx\d+ \{", src, re.M)) == mech.R
    assert src.count("asm volatile") == (mech.R + 3) // 4      # one barrier per group of four
    assert "advance_body<%d, true, rde::RhsOf<rde::jit::Reactions>, rde::kMethodRodas3>" % mech.K in src
    # ln A and E/R stay run-time data (parameter updates need no recompilation)
    assert src.count("return x.lnA;") == mech.R and src.count("return x.EaR;") == mech.R


def test_falloff_and_efficiencies_compile():
    mech = synth.isomer_mechanism(kind="TROE", reversible=True, A=3e5, b=0.3, E=40.0,
                                  low=(4e12, -0.5, 10.0), troe=(0.4, 300.0, 1800.0, 5000.0))
    mech.reactions[0].eff = {"X2": 2.0, "A": 0.7}
    src = _compile(mech.to_text())["source"]
    # alpha - 1 for X2 (index 2) and A (index 0), in the order they were given
    assert "M += 0x1p+0 * L[S::C + 2];" in src
    assert "M += -0x1.3333333333334p-2 * L[S::C + 0];" in src
    assert "has_T2() const { return 1; }" in src
    assert "troe_a() const { return 0x1.999999999999ap-2; }" in src


def test_ros2_kernels_compile():
    """The ROS2 forward kernels are a separate source: the same reaction descriptors, the
    integrator template instantiated for the two-stage method."""
    mech = synth.h2_air_mechanism(16105)
    r0 = _compile(mech.to_text(), 0)
    r2 = _compile(mech.to_text(), 2)
    assert r2["cubin_bytes"] > 0
    assert "advance_body<%d, false, rde::RhsOf<rde::jit::Reactions>, rde::kMethodRos2>" % mech.K in r2["source"]
    body = lambda s: s[:s.index("extern \"C\"")]
    assert body(r0["source"]) == body(r2["source"])


def test_compile_part_is_checked():
    library()
    with pytest.raises(rde_chem.RdeError) as e:
        rde_chem.rde_selftest_jit_compile(synth.h2_air_mechanism(16105).to_text(), 4)
    assert e.value.code == -2      # RDE_ERR_ARG


def test_wide_kernel_compiles():
    """The wide 256-thread queue kernel (part 3) compiles: RODAS3 over the same generated
    reactions, with the CTA width as the kernel body's template argument."""
    mech = synth.h2_air_mechanism(16105)
    r = _compile(mech.to_text(), 3)
    assert r["cubin_bytes"] > 0
    assert "rde_jit_queue_w" in r["source"]
    assert "rde::kMethodRodas3, 256>(a);" in r["source"]
