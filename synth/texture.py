"""Seeded textures and 8-bit grey-level images for the feature-matching inputs.

Section 2.1 detects ORB features in the template image and in every live image and matches
them; the paper's laparoscopy videos are not available, so the surface of a synthetic scene
(scene.py) is given a texture: a base grey level plus overlapping axis-aligned rectangles of
random contrast, defined on the surface's lateral coordinates (x, y) in mm, so that it moves
and deforms with the surface.  An image is that texture seen through each pixel (the template
camera, or the live camera after the frame's deformation and motion), rounded to 8 bits, 0 where
the pixel sees no surface.  The binary-test pattern of the descriptor (256 point pairs, drawn
once from a seed) is also made here: it is a random input both implementations receive.

Nothing here detects, describes or matches features.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .scene import Scene, make_scene, raycast_template, render_target


@dataclasses.dataclass
class Texture:
    base: float
    rect: np.ndarray     # (R, 4) x0, y0, x1, y1 (mm)
    val: np.ndarray      # (R,) grey-level offset inside each rectangle

    def eval(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        g = np.full(np.shape(x), self.base, dtype=np.float64)
        for (x0, y0, x1, y1), v in zip(self.rect, self.val):
            g = g + v * ((x >= x0) & (x < x1) & (y >= y0) & (y < y1))
        return g


def random_texture(rng: np.random.Generator, n_rect: int = 600, width_mm: float = 110.0,
                   aspect: float = 0.75) -> Texture:
    half_w = width_mm / 2.0
    half_h = half_w * aspect
    c = np.stack([rng.uniform(-half_w, half_w, n_rect), rng.uniform(-half_h, half_h, n_rect)], 1)
    size = rng.uniform(1.5, 8.0, (n_rect, 2))
    rect = np.concatenate([c - size / 2, c + size / 2], axis=1)
    val = rng.uniform(-70.0, 70.0, n_rect)
    return Texture(128.0, rect, val)


def to_u8(g: np.ndarray, seen: np.ndarray) -> np.ndarray:
    return np.where(seen, np.clip(np.rint(g), 0, 255), 0).astype(np.uint8)


def orb_pattern(seed: int, n: int = 256, sigma: float = 31.0 / 5.0, radius: float = 13.0):
    """n point pairs (ax, ay, bx, by), each point from an isotropic Gaussian of std sigma,
    redrawn until it lies in the disc of the given radius (so any rotation stays inside)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((n, 4))
    for i in range(n):
        for j in range(2):
            while True:
                p = rng.normal(0.0, sigma, 2)
                if p[0] * p[0] + p[1] * p[1] <= radius * radius:
                    break
            out[i, 2 * j:2 * j + 2] = p
    return out


@dataclasses.dataclass
class TexturedScene:
    scene: Scene
    texture: Texture
    template_image: np.ndarray     # (H, W) uint8
    images: list                   # (H, W) uint8 per frame
    live_xy: list                  # (H, W, 2) surface coordinates seen by each live pixel


def make_textured_scene(cfg, seed: int, n_frames: int | None = None, f64: bool = False,
                        **kw) -> TexturedScene:
    """The scene of make_scene(cfg, seed) (same geometry and matches) plus a texture drawn from
    a second seeded stream and the template / live images it produces."""
    sc = make_scene(cfg, seed, n_frames=n_frames, f64=f64, **kw)
    rng = np.random.default_rng([seed, 0x7E47])
    tex = random_texture(rng)
    tdepth, X0 = raycast_template(sc.hf, sc.W, sc.H)
    timg = to_u8(tex.eval(X0[..., 0], X0[..., 1]), tdepth > 0)
    images, xys = [], []
    for fr in sc.frames:
        _, x, y = render_target(sc.hf, fr.motion, sc.W, sc.H, return_xy=True)
        images.append(to_u8(tex.eval(x, y), np.asarray(fr.depth) > 0))
        xys.append(np.stack([x, y], axis=-1))
    return TexturedScene(sc, tex, timg, images, xys)
