"""Initial planes on the device (Sec. 3.1).

The paper starts each plane at a point of the coarse scene geometry with its
rotation from the local surface and all four radii at half the distance to the
nearest other plane centre.  The seeded point sets come from
``scenes`` (surface points of a synthetic room, or the degraded monocular-style
maps); the radii come from the library's exact nearest-neighbour kernel
``ps_nn_distance``, so a start for thousands of planes costs a few launches.
"""
from __future__ import annotations

import torch

from . import binding as B
from . import scenes as S

R_LO, R_HI = 0.02, 2.0          # radii kept in [2 cm, 2 m] (the host generators use the same)


def nn_radii(centers: torch.Tensor, scale: float = 0.5, r_lo: float = R_LO,
             r_hi: float = R_HI) -> torch.Tensor:
    """[n, 4] radii clamp(scale x nearest-other-centre distance, r_lo, r_hi) of
    centres [n, 3] (device f32), by ps_nn_distance."""
    c = centers.contiguous().float()
    radii = torch.empty((c.shape[0], 4), dtype=torch.float32, device=c.device)
    if c.shape[0] > 0:
        B.ps_nn_distance(c, radii=radii, scale=scale, r_lo=r_lo, r_hi=r_hi)
    return radii


def _with_radii(p: S.Planes, device, scale: float) -> S.Planes:
    c = torch.from_numpy(p.center).to(device)
    p.radii[:] = nn_radii(c, scale).cpu().numpy()
    return p


def surface_start(room: S.Room, n: int, seed: int, device="cuda", scale: float = 0.5) -> S.Planes:
    """n planes at random surface points of the room, random orientation, radii
    scale x nearest-centre distance (computed on the device)."""
    return _with_radii(S.surface_init(room, n, seed), device, scale)


def mono_start(room: S.Room, depth, normal, n: int, seed: int, device="cuda",
               scale: float = 0.5, **kw) -> S.Planes:
    """The monocular-style start of Sec. 3.1 (scenes.mono_points: centres
    back-projected from degraded depth, normals from degraded normal maps), with
    radii scale x nearest-centre distance computed on the device."""
    return _with_radii(S.mono_points(room, depth, normal, n, seed, **kw), device, scale)
