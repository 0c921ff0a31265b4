"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Nothing here computes any step of the deformation solve; see scene.py.
"""
from .scene import (CONFIGS, Config, Frame, Scene, control_point_pixels, intrinsics_for,
                    make_scene, seed_for)
from .texture import TexturedScene, make_textured_scene, orb_pattern

__all__ = ["CONFIGS", "Config", "Frame", "Scene", "control_point_pixels", "intrinsics_for",
           "make_scene", "seed_for", "TexturedScene", "make_textured_scene", "orb_pattern"]
