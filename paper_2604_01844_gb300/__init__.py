"""GB300 (sm_103a) Gaussian-splatting CT hot path of FaCT-GS (arXiv 2604.01844).

The compute runs in libgsct (C ABI: include/gsct.h, CUDA sources under csrc/); this package is
its thin Python binding.  Build it with paper_2604_01844_gb300.build.build() (or
__graft_entry__.build()).
"""
from . import binding
from .binding import GsError
from .projector import BatchProjector, Projector, ProjectFunction, project, views_to_device
from .voxelizer import BatchVoxelizer, Voxelizer, VoxelizeFunction, voxelize

__all__ = ["binding", "GsError", "BatchProjector", "Projector", "ProjectFunction", "project", "views_to_device",
           "BatchVoxelizer", "Voxelizer", "VoxelizeFunction", "voxelize"]
