"""Failure detection without a fault: the bounded waits of the library's kernels.  A wait on an
mbarrier that nothing completes must give up after its poll limit and report it, so that a lost
copy ends in SWE_ERR_TIMEOUT rather than a hung GPU, and the context must stay usable."""
import numpy as np
import pytest

from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def test_a_wait_nothing_completes_gives_up_and_the_context_stays_usable():
    assert swe.swe_probe_bounded_wait(2000, 0) is True          # nobody arrives: the wait gives up
    assert swe.swe_probe_bounded_wait(2000, 1) is False         # one arrival completes the phase
    assert swe.swe_probe_bounded_wait(1, 0) is True
    # the context still runs the tile step, whose copies use the same waits
    w = W.partial_dam_break(nx=30, ny=14, spacing=1.0, n_gauss=8, seed=3)
    m = swe.Mesh.from_workload(w)
    a = swe.State.from_workload(m, swe.swe_params_default("muscl", "fp64", kernel="fused"), w)
    b = swe.State.from_workload(m, swe.swe_params_default("muscl", "fp64", kernel="split"), w)
    a.step(5, 0.9)
    b.step(5, 0.9)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    a.close()
    b.close()
    m.close()


def test_bad_arguments_are_rejected():
    for polls in (0, (1 << 22) + 1):
        with pytest.raises(swe.SweError) as e:
            swe.swe_probe_bounded_wait(polls, 0)
        assert e.value.code == -1
