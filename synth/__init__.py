"""Seeded synthetic inputs shared by the tests, the benchmark and the
oracle's test harness: cone-beam geometries and voxel volumes.  This module
holds none of the projector's arithmetic."""
from .geometry import (ConeGeometry, VolumeGeometry, circular, cone_angle_geometry,  # noqa: F401
                       covering_pitch, c1_geometry, c2_geometry, c3_geometry, c4_geometry,
                       scaled_c2_geometry, random_geometry, exact_cos_sin, BatchProblemSpec,
                       c5_manifest, small_batch_manifest)
from .phantom import (SHEPP_LOGAN_SHAPED, ellipsoids_world, voxelize, random_field,  # noqa: F401
                      gaussian_field, build as build_phantom)
