"""save_checkpoint / load_checkpoint on the host: the file round-trips every parameter group,
Adam's moments, the seed, the iteration and the step number, and refuses a scene of another
shape.  (The GPU test resumes a real optimisation from one and compares the next iteration.)"""
import pytest
import torch

from paper_2404_09758_gb300 import load_checkpoint, save_checkpoint


class _FakeScene:
    def __init__(self, shapes, seed):
        g = torch.Generator().manual_seed(seed)
        self.groups = [torch.rand(*s, generator=g) for s in shapes]
        self.n_params = sum(x.numel() for x in self.groups)

    def param_groups(self):
        return self.groups


SHAPES = [(10, 3), (4, 5, 3), (2, 2, 1)]


def test_round_trip(tmp_path):
    a = _FakeScene(SHAPES, 1)
    m, v = torch.rand(a.n_params), torch.rand(a.n_params)
    path = tmp_path / "ck.pt"
    save_checkpoint(path, a, seed=77, it=4_000_000_000, t=12, m=m, v=v)
    b = _FakeScene(SHAPES, 2)
    m2, v2 = torch.zeros(a.n_params), torch.zeros(a.n_params)
    assert load_checkpoint(path, b, m=m2, v=v2) == (77, 4_000_000_000, 12)
    for x, y in zip(a.groups, b.groups):
        assert torch.equal(x, y)
    assert torch.equal(m, m2) and torch.equal(v, v2)


def test_without_moments(tmp_path):
    a = _FakeScene(SHAPES, 3)
    save_checkpoint(tmp_path / "sgd.pt", a, seed=1, it=2, t=3)
    m = torch.full((a.n_params,), 5.0)
    assert load_checkpoint(tmp_path / "sgd.pt", _FakeScene(SHAPES, 4), m=m) == (1, 2, 3)
    assert torch.all(m == 5.0)  # the file has no m: the buffer is left alone


def test_other_scene_or_file_is_refused(tmp_path):
    a = _FakeScene(SHAPES, 5)
    save_checkpoint(tmp_path / "ck.pt", a, seed=1, it=0, t=1)
    with pytest.raises(ValueError):
        load_checkpoint(tmp_path / "ck.pt", _FakeScene([(10, 3), (4, 5, 3)], 6))
    with pytest.raises(ValueError):
        load_checkpoint(tmp_path / "ck.pt", _FakeScene([(11, 3), (4, 5, 3), (2, 2, 1)], 6))
    torch.save({"something": 1}, tmp_path / "other.pt")
    with pytest.raises(ValueError):
        load_checkpoint(tmp_path / "other.pt", a)
    with pytest.raises(ValueError):
        save_checkpoint(tmp_path / "no_t.pt", a, seed=1, it=0)
