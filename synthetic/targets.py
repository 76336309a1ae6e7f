"""Seeded synthetic targets and geometries for the SiPO projection LP.

This module only draws shapes: target dose fields f_T (binary: 1 inside the
part, 0 outside; or graded: one prescribed level per part) and angle lists. It holds none of the method's arithmetic
(no projector, no LP, no solver), so both the CPU oracle and the CUDA path may
consume what it produces.

Layouts follow the solver's convention: a volume is a C-contiguous float32
array indexed [y][x][z] (z, the rotation axis, is the fastest index); a 2-D
slice is the same with nz = 1.  Voxel centres sit at i - (n - 1)/2.

The paper measures on a binary logo (Sec. 3.1) and a 3-D "Thinker" model
(Sec. 3.4), neither of which is available; these generators stand in for them
with binary parts of matched scale.  The grayscale experiment of Sec. 3.3
(one response level per character of the logo) is stood in for by discs with
one level each.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "uniform_angles",
    "discs_2d",
    "graded_discs_2d",
    "csg_3d",
    "lattice_3d",
    "Workload",
    "workload",
    "sweep_workloads",
]


def uniform_angles(n_angles: int, span: float = math.pi) -> np.ndarray:
    """n_angles uniformly spaced angles k*span/n_angles, k = 0..n-1 (float64, rad)."""
    return np.arange(n_angles, dtype=np.float64) * (span / n_angles)


def _centred(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.float64) - (n - 1) / 2.0


def discs_2d(n: int = 64, n_discs: int = 3, r_range=(6.0, 14.0),
             container_radius: float = 28.0, seed: int = 1) -> np.ndarray:
    """Union of `n_discs` discs on an n x n grid, returned as [n][n][1] float32.

    Radii are uniform in r_range; each whole disc lies inside the disc of radius
    `container_radius` about the grid centre (centre radius <= container - r).
    """
    rng = np.random.default_rng(seed)
    c = _centred(n)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    f = np.zeros((n, n), dtype=bool)
    for _ in range(n_discs):
        r = rng.uniform(*r_range)
        rho = (container_radius - r) * math.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        cx, cy = rho * math.cos(phi), rho * math.sin(phi)
        f |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    return f.astype(np.float32)[:, :, None].copy()


def graded_discs_2d(n: int = 64, levels=(1.0, 0.7, 0.45), r_range=(6.0, 14.0),
                    container_radius: float = 28.0, seed: int = 1) -> np.ndarray:
    """Discs with one prescribed level each (a multi-level grayscale target),
    returned as [n][n][1] float32.

    Disc k has level levels[k] and is placed like a disc of `discs_2d`; where
    discs overlap the later one wins, so every gel voxel carries exactly one
    of the levels.
    """
    rng = np.random.default_rng(seed)
    c = _centred(n)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    f = np.zeros((n, n), dtype=np.float32)
    for level in levels:
        r = rng.uniform(*r_range)
        rho = (container_radius - r) * math.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        cx, cy = rho * math.cos(phi), rho * math.sin(phi)
        f[(xx - cx) ** 2 + (yy - cy) ** 2 <= r * r] = np.float32(level)
    return f[:, :, None].copy()


def _random_unit(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _prim_mask(kind, centre, axis, dims, n, nz, pad):
    """Boolean mask of one primitive, evaluated only on its bounding box.

    Returns (slices, mask) with mask shaped like the box.  Coordinates are
    (x, y, z) voxel-centre offsets from the grid centre.
    """
    extent = dims["bound"] + pad
    cy_, cx_, cz_ = (n - 1) / 2.0, (n - 1) / 2.0, (nz - 1) / 2.0
    lo = [max(0, int(math.floor(centre[1] + cy_ - extent))),
          max(0, int(math.floor(centre[0] + cx_ - extent))),
          max(0, int(math.floor(centre[2] + cz_ - extent)))]
    hi = [min(n, int(math.ceil(centre[1] + cy_ + extent)) + 1),
          min(n, int(math.ceil(centre[0] + cx_ + extent)) + 1),
          min(nz, int(math.ceil(centre[2] + cz_ + extent)) + 1)]
    if any(h <= l for l, h in zip(lo, hi)):
        return None, None
    y = np.arange(lo[0], hi[0]) - cy_ - centre[1]
    x = np.arange(lo[1], hi[1]) - cx_ - centre[0]
    z = np.arange(lo[2], hi[2]) - cz_ - centre[2]
    Y, X, Z = np.meshgrid(y, x, z, indexing="ij")
    if kind == "sphere":
        m = X * X + Y * Y + Z * Z <= dims["r"] ** 2
    else:
        along = X * axis[0] + Y * axis[1] + Z * axis[2]
        perp2 = X * X + Y * Y + Z * Z - along * along
        if kind == "cylinder":
            m = (perp2 <= dims["r"] ** 2) & (np.abs(along) <= dims["half_len"])
        else:  # torus with normal `axis`
            ring = np.sqrt(np.maximum(perp2, 0.0)) - dims["R"]
            m = ring * ring + along * along <= dims["r"] ** 2
    sl = (slice(lo[0], hi[0]), slice(lo[1], hi[1]), slice(lo[2], hi[2]))
    return sl, m


def csg_3d(n: int = 256, nz: int | None = None, vial_radius: float = 120.0,
           band_width: int = 10, seed: int = 2, n_prims=(4, 8),
           feature=(10.0, 60.0), kinds=("sphere", "cylinder", "torus"),
           p_add: float = 0.75) -> np.ndarray:
    """Seeded CSG of spheres, cylinders and tori inside a vial, [n][n][nz] float32.

    U{n_prims} primitives, each additive with probability p_add (the first is
    always additive) or subtractive, applied in sequence.  Diameters (sphere
    and cylinder) and tube diameters (torus) are uniform in `feature`.  The
    result is clipped to r_xy <= vial_radius - band_width and to
    z in [band_width, nz-1-band_width]; an empty result is redrawn.
    """
    nz = n if nz is None else nz
    inner = vial_radius - band_width
    for attempt in range(64):
        rng = np.random.default_rng(seed + 7919 * attempt)
        f = np.zeros((n, n, nz), dtype=bool)
        k = int(rng.integers(n_prims[0], n_prims[1] + 1))
        zhalf = max(1.0, (nz - 1) / 2.0 - band_width)
        for i in range(k):
            kind = kinds[int(rng.integers(len(kinds)))]
            d = rng.uniform(*feature)
            rho = 0.75 * inner * math.sqrt(rng.uniform())
            phi = rng.uniform(0, 2 * math.pi)
            centre = (rho * math.cos(phi), rho * math.sin(phi),
                      rng.uniform(-0.75 * zhalf, 0.75 * zhalf))
            axis = _random_unit(rng)
            if kind == "sphere":
                dims = {"r": d / 2, "bound": d / 2}
            elif kind == "cylinder":
                half_len = rng.uniform(d / 2, 2.0 * d)
                dims = {"r": d / 2, "half_len": half_len,
                        "bound": math.hypot(d / 2, half_len)}
            else:
                R = rng.uniform(d / 2 + 2.0, d / 2 + feature[1] / 2)
                dims = {"r": d / 2, "R": R, "bound": R + d / 2}
            sl, m = _prim_mask(kind, centre, axis, dims, n, nz, 1.0)
            if sl is None:
                continue
            if i == 0 or rng.uniform() < p_add:
                f[sl] |= m
            else:
                f[sl] &= ~m
        c = _centred(n)
        yy, xx = np.meshgrid(c, c, indexing="ij")
        f &= ((xx * xx + yy * yy) <= inner * inner)[:, :, None]
        zi = np.arange(nz)
        f &= ((zi >= band_width) & (zi <= nz - 1 - band_width))[None, None, :]
        if f.any():
            return f.astype(np.float32)
    raise RuntimeError("could not draw a non-empty CSG target")


def lattice_3d(n: int = 512, vial_radius: float = 240.0, band_width: int = 10,
               cells: int = 4, seed: int = 5, width=(6.0, 12.0)) -> np.ndarray:
    """Lattice of cells^3 interlocking tori joined by struts, [n][n][n] float32.

    The lattice fills the largest cube inside r_xy <= vial_radius - band_width.
    Each cell holds a torus whose normal cycles x, y, z with the cell parity,
    so neighbouring rings interlock; cylinders (struts) join neighbouring cell
    centres.  Tube and strut widths are uniform in `width`.
    """
    rng = np.random.default_rng(seed)
    inner = vial_radius - band_width
    half = min(inner / math.sqrt(2.0), (n - 1) / 2.0 - band_width) - 4.0
    cell = 2 * half / cells
    f = np.zeros((n, n, n), dtype=bool)
    axes = [np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])]
    centres = {}
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                c = (-half + (i + 0.5) * cell, -half + (j + 0.5) * cell,
                     -half + (k + 0.5) * cell)
                centres[(i, j, k)] = c
                d = rng.uniform(*width)
                R = 0.3 * cell
                dims = {"r": d / 2, "R": R, "bound": R + d / 2}
                sl, m = _prim_mask("torus", c, axes[(i + j + k) % 3], dims, n, n, 1.0)
                if sl is not None:
                    f[sl] |= m
    for (i, j, k), c in centres.items():
        for di, dj, dk in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            nb = (i + di, j + dj, k + dk)
            if nb not in centres:
                continue
            c2 = centres[nb]
            mid = tuple((a + b) / 2 for a, b in zip(c, c2))
            axis = np.array([c2[0] - c[0], c2[1] - c[1], c2[2] - c[2]])
            length = float(np.linalg.norm(axis))
            d = rng.uniform(*width)
            dims = {"r": d / 2, "half_len": length / 2,
                    "bound": math.hypot(d / 2, length / 2)}
            sl, m = _prim_mask("cylinder", mid, axis / length, dims, n, n, 1.0)
            if sl is not None:
                f[sl] |= m
    return f.astype(np.float32)


@dataclass
class Workload:
    """One LP instance: geometry, target and case parameters (plain data)."""
    name: str
    n: int
    nz: int
    n_angles: int
    n_det: int
    angles: np.ndarray
    target: np.ndarray            # [n][n][nz] float32
    case: int                     # 0 general, 1 case 1, 2 case 2
    vial_radius: float = 0.0
    mu: float = 0.0
    psf_sigma: tuple = (0.0, 0.0, 0.0)
    psf_trunc: float = 4.0
    band_width: int = 10
    w1: float = 1.0
    w2: float = 1.0
    tol_lo: float = 0.05
    tol_hi: float = 0.05
    inhibit_ratio: float = 0.8
    kkt_tol: float = 1e-4
    extra: dict = field(default_factory=dict)


def workload(name: str, seed: int | None = None) -> Workload:
    """The named measurement workloads.

    - "disc64": 64x64 slice, 96 angles over [0, pi), 91 bins, 3 discs, Case 1
      (delta = 0.05), no vial/attenuation/blur, KKT 1e-6, FP64.
    - "csg256": 256^3, 360 angles, 256 bins, CSG target in a radius-120 vial,
      Case 2 (ratio 0.8), no attenuation or blur, FP32.
    - "csg256_blur": as csg256 with mu = 0.005/voxel and PSF sigma (1.5,1.5,2.5).
    - "lattice512": 512^3, 720 angles, 512 bins, mu 0.0025, sigma (2,2,3),
      radius-240 vial, Case 2, BF16 storage.
    Smaller variants ("csg64", "csg128") share the csg recipe at reduced size.
    """
    if name == "disc64":
        s = 1 if seed is None else seed
        return Workload(name, 64, 1, 96, 91, uniform_angles(96),
                        discs_2d(64, seed=s), case=1, band_width=10,
                        tol_lo=0.05, tol_hi=0.05, kkt_tol=1e-6)
    if name.startswith("csg"):
        blur = name.endswith("_blur")
        n = int(name[3:].split("_")[0])
        s = 2 if seed is None else seed
        n_ang = {256: 360}.get(n, max(16, int(round(n * 360 / 256))))
        scale = n / 256.0
        vial = 120.0 * scale
        bw = max(2, int(round(10 * scale)))
        tgt = csg_3d(n, vial_radius=vial, band_width=bw, seed=s,
                     feature=(10.0 * scale, 60.0 * scale))
        wl = Workload(name, n, n, n_ang, n, uniform_angles(n_ang), tgt, case=2,
                      vial_radius=vial, band_width=bw, inhibit_ratio=0.8)
        if blur:
            wl.mu = 0.005 / scale
            wl.psf_sigma = (1.5, 1.5, 2.5)
        return wl
    if name == "lattice512":
        s = 5 if seed is None else seed
        return Workload(name, 512, 512, 720, 512, uniform_angles(720),
                        lattice_3d(512, seed=s), case=2, vial_radius=240.0,
                        mu=0.0025, psf_sigma=(2.0, 2.0, 3.0), band_width=10,
                        inhibit_ratio=0.8)
    raise KeyError(name)


def sweep_workloads(n_problems: int = 32, seed: int = 100,
                    sizes=(64, 192), angles=(180, 720)) -> list[Workload]:
    """The batched sweep: independent LPs on seeded cubes with sphere/torus targets.

    Sizes are multiples of 16 in `sizes`, angle counts uniform in `angles`.
    The first half are Case 1 with delta cycling over {0.02, 0.04, ..., 0.20};
    the second half Case 2 with the ratio cycling over {0.60, 0.65, ..., 0.90}.
    """
    deltas = [0.02 * (i + 1) for i in range(10)]
    ratios = [0.60 + 0.05 * i for i in range(7)]
    out = []
    half = n_problems // 2
    for p in range(n_problems):
        rng = np.random.default_rng(seed + p)
        n = int(rng.integers(sizes[0] // 16, sizes[1] // 16 + 1)) * 16
        n_ang = int(rng.integers(angles[0], angles[1] + 1))
        vial = 0.47 * n
        bw = max(2, int(round(10 * n / 256)))
        tgt = csg_3d(n, vial_radius=vial, band_width=bw, seed=seed + 1000 + p,
                     n_prims=(1, 3), feature=(0.08 * n, 0.3 * n),
                     kinds=("sphere", "torus"), p_add=1.0)
        if p < half:
            wl = Workload(f"sweep{p}", n, n, n_ang, n, uniform_angles(n_ang), tgt,
                          case=1, vial_radius=vial, band_width=bw,
                          tol_lo=deltas[p % 10], tol_hi=deltas[p % 10])
        else:
            wl = Workload(f"sweep{p}", n, n, n_ang, n, uniform_angles(n_ang), tgt,
                          case=2, vial_radius=vial, band_width=bw,
                          inhibit_ratio=ratios[(p - half) % 7])
        out.append(wl)
    return out
