"""Host logic of the batched path (no GPU): the autotuner's search and the
batch signature used to cache its choices."""
import pytest

torch = pytest.importorskip("torch")


def test_coordinate_search_finds_separable_optimum():
    from paper_2311_15038_gb300 import BatchTuning
    from paper_2311_15038_gb300.batch import coordinate_search
    calls = []

    def cost(t):
        calls.append(t)
        return abs(t.warp_w - 16) + abs(t.chunk - 4) * 0.5 + (0.2 if t.ctas_per_sm == 0 else 0.0)

    best = coordinate_search(cost)
    assert best == BatchTuning(16, 4, 2)
    assert len(calls) == 4 + 5 + 2


def test_coordinate_search_ties_keep_first():
    from paper_2311_15038_gb300 import BatchTuning
    from paper_2311_15038_gb300.batch import coordinate_search
    assert coordinate_search(lambda t: 1.0) == BatchTuning(4, 1, 0)


def test_signature_depends_on_levels_and_views():
    from paper_2311_15038_gb300 import Slicemap, View
    from paper_2311_15038_gb300.batch import _signature
    a = Slicemap((64, 64, 64), [(32, 32, 32)], [(8, 4)], [torch.empty(1)], 8, torch.uint8)
    b = Slicemap((64, 64, 64), [(16, 16, 16)], [(4, 4)], [torch.empty(1)], 8, torch.uint8)
    luts = torch.zeros(1, 256, 4)
    v = [View(0.0, 0.0, 32, 32)]
    assert _signature([a], v, [0], luts) == _signature([a], v, [0], luts)
    assert _signature([a], v, [0], luts) != _signature([b], v, [0], luts)
    assert _signature([a], v, [0], luts) != _signature([a], v * 2, [0, 0], luts)
