"""The product path has no CPU fallback: without the CUDA library, or with host tensors, every
compute entry point raises instead of computing."""
import pytest
import torch

import synth


@pytest.fixture
def missing_library(monkeypatch):
    from paper_2604_01844_gb300 import binding

    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", "/nonexistent/libgsct.so")
    return binding


def test_missing_library_raises(missing_library):
    import paper_2604_01844_gb300 as g

    B = missing_library
    with pytest.raises(B.GsError, match="not built"):
        B.lib()
    mr, sc, qt = [torch.from_numpy(a) for a in synth.gaussians(0, 10)]
    proj = g.Projector(synth.cone_views(2, 16, 16), 16, 16, device="cpu")
    with pytest.raises(B.GsError):
        proj.count_evals(mr, sc, qt)


def test_host_tensors_are_rejected(missing_library):
    import paper_2604_01844_gb300 as g

    mr, sc, qt = [torch.from_numpy(a) for a in synth.gaussians(0, 10)]
    with pytest.raises(ValueError, match="CUDA"):
        g.Projector(synth.cone_views(2, 16, 16), 16, 16, device="cpu").forward(mr, sc, qt)
    with pytest.raises(ValueError, match="CUDA"):
        g.Voxelizer(synth.cube_grid(16), device="cpu").forward(mr, sc, qt)
