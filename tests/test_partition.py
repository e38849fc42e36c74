"""Sub-domains with two halo layers (Sec. 6.4), host side: every list against a brute force over the
exported adjacency (no GPU needed)."""
import numpy as np
import pytest

from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe
from paper_2307_16758_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def _brute(nbr, a, b):
    """halo1, halo2 of the owned range [a, b) from the adjacency."""
    owned = set(range(a, b))
    h1 = {int(j) for c in range(a, b) for j in nbr[c] if j >= 0 and j not in owned}
    h2 = {int(j) for c in h1 for j in nbr[c] if j >= 0 and j not in owned and j not in h1}
    return sorted(h1), sorted(h2)


@pytest.mark.parametrize("n_parts", [1, 2, 5, 16])
def test_halo_layers_boundary_and_interior(n_parts):
    w = W.partial_dam_break(nx=40, ny=20, spacing=1.0, n_gauss=10, seed=4)
    m = swe.Mesh.from_workload(w, "morton")
    nbr = m.export()["nbr"]
    part = swe.Partition(m, n_parts)
    n = m.n
    starts, halos = [], []
    for p in range(n_parts):
        a, b, n1, n2, nb = part.info(p)
        starts.append((a, b))
        h1, h2, bnd = part.export(p)
        e1, e2 = _brute(nbr, a, b)
        assert h1.tolist() == e1 and h2.tolist() == e2
        halos.append(set(e1) | set(e2))
    # contiguous, covering, of equal size within one cell
    assert starts[0][0] == 0 and starts[-1][1] == n
    assert all(starts[p][1] == starts[p + 1][0] for p in range(n_parts - 1))
    sizes = [b - a for a, b in starts]
    assert max(sizes) - min(sizes) <= 1
    # boundary = owned cells that another part holds in a halo
    for p, (a, b) in enumerate(starts):
        others = set().union(*[halos[q] for q in range(n_parts) if q != p]) if n_parts > 1 else set()
        want = sorted(c for c in range(a, b) if c in others)
        assert part.export(p)[2].tolist() == want
    if n_parts == 1:
        assert part.info(0)[2:] == (0, 0, 0)
    part.close()
    m.close()


def test_bad_part_counts_are_rejected():
    w = W.dam_break_1d(10, 2, 10.0, 2.0)
    m = swe.Mesh.from_workload(w)
    for k in (0, -1, m.n + 1, 2000):
        with pytest.raises(swe.SweError) as e:
            swe.Partition(m, k)
        assert e.value.code == -1
    m.close()


def test_one_cell_per_part():
    """The degenerate split: every cell its own sub-domain (halo1 = its neighbours, every cell on a
    boundary list)."""
    w = W.dam_break_1d(4, 2, 4.0, 2.0)
    m = swe.Mesh.from_workload(w, "morton")
    nbr = m.export()["nbr"]
    n = m.n
    part = swe.Partition(m, n)
    for p in range(n):
        a, b, n1, n2, nb = part.info(p)
        assert (a, b) == (p, p + 1)
        h1, h2, bnd = part.export(p)
        e1, e2 = _brute(nbr, a, b)
        assert h1.tolist() == e1 and h2.tolist() == e2
        assert bnd.tolist() == [p]
    part.close()
    m.close()
