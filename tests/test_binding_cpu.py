"""Host-side logic of the Python binding that needs no GPU: the column-wise
conversion of a batch of C statistics records."""
import ctypes

import pytest

torch = pytest.importorskip("torch")


def test_batched_stats_conversion_matches_per_record_path():
    import paper_2101_06385_gb300 as m

    B = 37
    st = (m._Stats * B)()
    for i in range(B):
        s = st[i]
        s.iterations = 20 + i % 7
        s.launches = 40
        s.converged_by = [1, 3, 4, 5][i % 4]
        s.e_min, s.e_max, s.trace, s.energy = -1.0 - i, 2.0 + i, 0.5 * i, -3.25 * i
        for k in range(s.iterations):
            s.sigma[k] = 1 if (k + i) % 3 else -1
            s.iderr[k] = 1.0 / (k + 1 + i)
        for k in range(s.launches):
            s.layer_ms[k] = 0.5 + k
            s.square_ms[k] = 0.25 + k
    many = m._stats_many(st, B)
    one = [m._stats(st[i], 1 if st[i].converged_by == 4 else 0) for i in range(B)]
    assert many == one
    assert many[3].converged_by == "bounds" and many[2].converged_by == "max_iter" and many[2].status == 1
    assert many[3].energy == pytest.approx(-9.75)


def test_record_layout_matches_header():
    """The ctypes mirror has the fields the C header declares, in order, with
    the energy field last."""
    import paper_2101_06385_gb300 as m

    names = [f[0] for f in m._Stats._fields_]
    assert names[-1] == "energy" and names[:2] == ["iterations", "converged_by"]
    assert ctypes.sizeof(m._Stats) % 8 == 0
