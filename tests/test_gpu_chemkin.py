"""A mechanism imported from CHEMKIN-II text loads through the C ABI, matches the
oracle on the imported text to the parity bounds, and advances like the mechanism it
was written from up to the format's rounding of the NASA-7 coefficients (9 digits:
the two are slightly different mechanisms, about 2e-9 apart in Y here)."""
import pytest

from gpu_util import assert_parity, library, run_gpu, run_oracle
from paper_2508_16105_gb300 import chemkin, rde_chem, synth

pytestmark = pytest.mark.gpu


def test_imported_mechanism_runs_on_the_gpu(h2mech):
    library()
    back = chemkin.read_chemkin(chemkin.write_chemkin(h2mech))
    cells = synth.uniform_cells(h2mech, 256, seed=1014)
    a = run_gpu(h2mech, cells, 1e-8, flags=rde_chem.RDE_LOAD_GENERIC)
    b = run_gpu(back, cells, 1e-8, flags=rde_chem.RDE_LOAD_GENERIC)
    assert (a["status"] == 0).all()
    assert_parity(b, run_oracle(back, cells, 1e-8))
    assert_parity(b, a, T_tol=1e-6, Y_tol=1e-8)
