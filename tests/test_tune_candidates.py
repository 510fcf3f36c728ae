"""The autotuner's launch candidates (host logic, no GPU): thread per cell on both
schedules, the 128-thread queue at every CTA count that fits, the wide 256-thread
queue kernel where the handle can build it, and the CTA-per-cell kernel."""
from paper_2508_16105_gb300 import rde_chem, tune

PLAIN, QUEUE, BLOCK = rde_chem.RDE_SCHED_PLAIN, rde_chem.RDE_SCHED_QUEUE, rde_chem.RDE_SCHED_BLOCK


def test_candidates_thread_per_cell_with_wide():
    c = tune.candidates(2, thread_per_cell=True, wide=True)
    assert dict(schedule=PLAIN, ctas_per_sm=0, threads_per_cta=128) in c
    assert [x["ctas_per_sm"] for x in c if x["schedule"] == QUEUE and x["threads_per_cta"] == 128] == [1, 2]
    assert dict(schedule=QUEUE, ctas_per_sm=0, threads_per_cta=256) in c
    assert c[-1] == dict(schedule=BLOCK, ctas_per_sm=0, threads_per_cta=0)
    assert len(c) == 5


def test_candidates_without_wide_or_thread_per_cell():
    c = tune.candidates(1, thread_per_cell=True, wide=False)
    assert all(x["threads_per_cta"] != 256 for x in c) and len(c) == 3
    # a mechanism only the CTA-per-cell kernel serves: one candidate
    assert tune.candidates(3, thread_per_cell=False, wide=True) == [dict(schedule=BLOCK, ctas_per_sm=0,
                                                                         threads_per_cta=0)]
    # at least one queue candidate even if no CTA count was reported
    assert [x for x in tune.candidates(0, True) if x["schedule"] == QUEUE][0]["ctas_per_sm"] == 1
