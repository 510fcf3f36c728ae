"""Autotuner: picks a valid launch from timed candidates and reuses its cache."""
import pytest

from gpu_util import library, to_dev
from paper_2508_16105_gb300 import rde_chem, synth, tune

pytestmark = pytest.mark.gpu


def test_tune_and_cache(tmp_path, monkeypatch):
    library()
    monkeypatch.setenv("RDE_TUNE_CACHE", str(tmp_path / "tune.json"))
    mech = synth.h2_air_mechanism(16105)
    cells = synth.field_cells(mech, 20000, seed=1002)
    m = rde_chem.Mechanism(mech.to_text())
    p, T, Y = to_dev(cells.p), to_dev(cells.T), to_dev(cells.Y)
    T0 = T.clone()
    r = tune.tune(m, mech.to_text(), p, T, Y, 5e-9, sample=4096)
    assert not r["cached"] and len(r["trials"]) >= 3
    assert r["sample"] == 20000      # raised to fill every lane of the GPU (capped at the cell count)
    assert rde_chem.RDE_SCHED_BLOCK in [t["schedule"] for t in r["trials"]]   # threads per cell: 1 or 128
    # nine species: one thread per cell beats 128 threads sharing one small cell
    assert r["schedule"] in (rde_chem.RDE_SCHED_PLAIN, rde_chem.RDE_SCHED_QUEUE)
    assert (T == T0).all()           # the caller's cells are not touched
    r2 = tune.tune(m, mech.to_text(), p, T, Y, 5e-9, sample=4096)
    assert r2["cached"] and r2["schedule"] == r["schedule"]
    info = rde_chem.rde_chem_kernel_info(m.handle)
    assert info["threads_per_cta"] == 128 and info["max_ctas_per_sm"] >= 1
    # CTA width: the 128-thread kernels and the wide 256-thread queue kernel are both timed
    assert 256 in [t["threads_per_cta"] for t in r["trials"]] and r["threads_per_cta"] in (0, 128, 256)
    m.close()
