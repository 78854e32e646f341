"""Checkpoint and resume of the reduced-volume fit (diff.Fitter), host side:
the saved state round-trips through torch.save, a fitter loaded from it holds
the same volume, transfer function, Adam moments and step count, and a state
saved for other views or another source is refused."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _fitter(views, src=(32, 32, 32), seed=0):
    from paper_2311_15038_gb300 import diff
    g = torch.Generator().manual_seed(seed)
    vol = torch.rand((8, 8, 8), generator=g)
    lut = torch.rand((16, 4), generator=g)
    targets = torch.zeros(sum(v.width * v.height * 4 for v in views))
    return diff.Fitter(vol, lut, views, src, targets)


def test_state_round_trip(tmp_path):
    import paper_2311_15038_gb300 as mctp
    views = [mctp.View(10.0 * k, 20.0, 12, 10, 0, 0.5) for k in range(3)]
    a = _fitter(views, seed=1)
    g = torch.Generator().manual_seed(9)
    for k in a._STATE:
        getattr(a, k).copy_(torch.rand(getattr(a, k).shape, generator=g))
    a.t = 17
    a.lr_vol = 3e-3
    path = tmp_path / "fit.pt"
    torch.save(a.state_dict(), path)
    b = _fitter(views, seed=2)
    b.load_state_dict(torch.load(path))
    for k in a._STATE:
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    assert b.t == 17 and b.lr_vol == 3e-3 and b.lr_lut == a.lr_lut


def test_state_for_other_views_is_refused():
    import paper_2311_15038_gb300 as mctp
    views = [mctp.View(0.0, 0.0, 12, 10, 0, 0.5)]
    state = _fitter(views).state_dict()
    other = _fitter([mctp.View(5.0, 0.0, 12, 10, 0, 0.5)])
    with pytest.raises(ValueError, match="views"):
        other.load_state_dict(state)
    with pytest.raises(ValueError, match="views"):
        _fitter(views, src=(32, 32, 31)).load_state_dict(state)
    bad = dict(state, vol=torch.zeros((4, 4, 4)))
    with pytest.raises(ValueError, match="shape"):
        _fitter(views).load_state_dict(bad)
