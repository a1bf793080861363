"""Seeded synthetic voxel geometries (solid masks) for the permeability solver.

This module only draws random numbers and rasterises shapes into ``uint8`` masks
(1 = solid, 0 = pore, C order ``[nz][ny][nx]``, x fastest).  It holds none of the
flow method's arithmetic, so both the CUDA path and the CPU oracle can take their
inputs from it.  Every generator takes an explicit seed and uses NumPy's
``Generator(PCG64(seed))``, which gives the same stream on every platform.

A voxel with integer index (x, y, z) has its centre at (x + 1/2, y + 1/2, z + 1/2);
a voxel belongs to a sphere (disk, tube) when the periodic (minimum-image)
distance from its centre to the shape is at most the radius.  The paper works on
binarised images with this voxel convention (Sec. 5.1); the shapes stand in for
its sphere packs (Sec. 6.3, 6.5), foam (Sec. 7.2) and precipitation cell (Sec. 7.3).
"""
from __future__ import annotations

import hashlib

import numpy as np

__all__ = [
    "rng",
    "mask_sha256",
    "porosity",
    "overlapping_spheres",
    "rsa_sphere_pack",
    "slit",
    "square_duct",
    "tube",
    "sc_sphere",
    "random_blocks",
    "voronoi_foam",
    "disk_cell",
    "clogging_sequence",
    "crops",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def mask_sha256(mask: np.ndarray) -> str:
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    h = hashlib.sha256()
    h.update(np.array(m.shape, dtype=np.int64).tobytes())
    h.update(m.tobytes())
    return h.hexdigest()


def porosity(mask: np.ndarray) -> float:
    return float(np.count_nonzero(mask == 0)) / mask.size


def _axis_offsets(c: float, reach: float, n: int):
    """Voxel indices whose centres lie within ``reach`` of coordinate ``c``
    (unwrapped), their wrapped indices and centre-to-c offsets."""
    lo = int(np.floor(c - reach - 0.5))
    hi = int(np.ceil(c + reach - 0.5))
    idx = np.arange(lo, hi + 1)
    d = (idx + 0.5) - c
    return np.mod(idx, n), d


def _paint_ball(mask: np.ndarray, centre, r: float) -> None:
    """Set to 1 every voxel whose centre is within r of ``centre`` (periodic)."""
    nz, ny, nx = mask.shape
    cx, cy, cz = centre
    ix, dx = _axis_offsets(cx, r, nx)
    iy, dy = _axis_offsets(cy, r, ny)
    iz, dz = _axis_offsets(cz, r, nz)
    d2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
    inside = d2 <= r * r
    if inside.any():
        sub = mask[np.ix_(iz, iy, ix)]
        sub |= inside.astype(np.uint8)
        mask[np.ix_(iz, iy, ix)] = sub


def overlapping_spheres(shape, radius: float, target_porosity: float, seed: int) -> np.ndarray:
    """Boolean model: spheres of one radius with centres uniform in the periodic box,
    added one at a time until the porosity first drops to ``target_porosity`` or below."""
    nz, ny, nx = shape
    g = rng(seed)
    mask = np.zeros(shape, dtype=np.uint8)
    n_solid_target = (1.0 - target_porosity) * mask.size
    while np.count_nonzero(mask) < n_solid_target:
        c = g.random(3) * np.array([nx, ny, nz], dtype=np.float64)
        _paint_ball(mask, c, radius)
    return mask


def _min_scaled_distance(shape, centres, radii, s_max: float) -> np.ndarray:
    """m(v) = min over spheres of |v - c_s| / r_s, evaluated where it is <= s_max
    (inf elsewhere).  Voxel v is solid at dilation factor s iff m(v) <= s."""
    nz, ny, nx = shape
    m = np.full(shape, np.inf, dtype=np.float64)
    for (cx, cy, cz), r in zip(centres, radii):
        reach = r * s_max
        ix, dx = _axis_offsets(cx, reach, nx)
        iy, dy = _axis_offsets(cy, reach, ny)
        iz, dz = _axis_offsets(cz, reach, nz)
        d = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) / r
        sub = m[np.ix_(iz, iy, ix)]
        np.minimum(sub, d, out=sub)
        m[np.ix_(iz, iy, ix)] = sub
    return m


def rsa_sphere_pack(shape, median: float, sigma: float, r_min: float, r_max: float,
                    target_porosity: float, seed: int, max_rejections: int = 20000,
                    attempts_per_sphere: int = 500, fill: float = 0.45, s_max: float = 1.6):
    """Consolidated random sphere pack.

    1. Radii r = median * exp(sigma * N(0, 1)) clipped to [r_min, r_max], drawn until
       their total sphere volume reaches ``fill`` x the box volume; sorted, largest
       first.
    2. Random sequential addition of non-overlapping spheres (periodic minimum
       image): each radius gets up to ``attempts_per_sphere`` random centres and is
       skipped if none fits; addition stops after ``max_rejections`` consecutive
       rejected trials (jamming) or when the radii run out.
    3. Non-overlapping addition jams well above porosity 0.38, so all radii are
       then dilated by one common factor s (overlaps allowed) chosen so that the
       porosity equals the target (to one voxel).

    Returns (mask, info) where info holds the centres, radii and the factor s.
    """
    nz, ny, nx = shape
    box = np.array([nx, ny, nz], dtype=np.float64)
    g = rng(seed)
    radii = []
    vol = 0.0
    while vol < fill * float(nx * ny * nz):
        r = float(np.clip(median * np.exp(sigma * g.standard_normal()), r_min, r_max))
        radii.append(r)
        vol += 4.0 / 3.0 * np.pi * r**3
    radii = np.sort(np.array(radii))[::-1]
    n_radii = len(radii)
    centres = np.zeros((n_radii, 3))
    acc_r = np.zeros(n_radii)
    n_acc = 0
    rejections = 0
    for r in radii:
        if rejections >= max_rejections:
            break
        for _ in range(attempts_per_sphere):
            c = g.random(3) * box
            if n_acc:
                d = centres[:n_acc] - c
                d -= box * np.round(d / box)
                ok = bool(np.all(np.einsum("ij,ij->i", d, d) >= (acc_r[:n_acc] + r) ** 2))
            else:
                ok = True
            if ok:
                centres[n_acc] = c
                acc_r[n_acc] = r
                n_acc += 1
                rejections = 0
                break
            rejections += 1
            if rejections >= max_rejections:
                break
    centres = centres[:n_acc]
    acc_r = acc_r[:n_acc]
    m = _min_scaled_distance(shape, centres, acc_r, s_max)
    n_fluid = int(round(target_porosity * m.size))
    flat = np.sort(m, axis=None)
    # solid iff m <= s; want exactly N - n_fluid solid voxels
    n_solid = m.size - n_fluid
    s = flat[n_solid - 1]
    if not np.isfinite(s) or s >= s_max:
        raise ValueError("dilation factor exceeds s_max; raise s_max")
    mask = (m <= s).astype(np.uint8)
    return mask, {"centres": centres, "radii": acc_r, "dilation": float(s)}


def slit(nx: int, h: int, period: int, nz: int = 1, axis_normal: int = 1) -> np.ndarray:
    """Plane channel: along the normal axis, ``h`` fluid layers followed by
    ``period - h`` solid layers; uniform along the other two axes."""
    prof = np.zeros(period, dtype=np.uint8)
    prof[h:] = 1
    if axis_normal == 1:
        return np.broadcast_to(prof[None, :, None], (nz, period, nx)).copy()
    if axis_normal == 0:
        return np.broadcast_to(prof[None, None, :], (nz, nx, period)).copy()
    return np.broadcast_to(prof[:, None, None], (period, nz, nx)).copy()


def square_duct(nx: int, a: int, period: int) -> np.ndarray:
    """Square duct of a x a fluid voxels along x in a period x period cross-section."""
    m = np.ones((period, period, nx), dtype=np.uint8)
    m[:a, :a, :] = 0
    return m


def tube(nx: int, radius: float, period: int) -> np.ndarray:
    """Circular tube along x: fluid where the distance from the voxel centre to the
    axis (at the centre of the period x period cross-section) is below ``radius``."""
    c = period / 2.0
    yy = np.arange(period) + 0.5 - c
    d2 = yy[:, None] ** 2 + yy[None, :] ** 2
    sec = (d2 >= radius * radius).astype(np.uint8)
    return np.broadcast_to(sec[:, :, None], (period, period, nx)).copy()


def sc_sphere(L: int, a: float) -> np.ndarray:
    """One sphere of radius ``a`` centred in a periodic L^3 cell (simple cubic array)."""
    m = np.zeros((L, L, L), dtype=np.uint8)
    _paint_ball(m, (L / 2.0, L / 2.0, L / 2.0), a)
    return m


def rotated_ellipsoid(n: int = 100, semi=(35.0, 10.0, 35.0), alpha_deg: float = 0.0) -> np.ndarray:
    """Anisotropy benchmark of Sec. 6: one solid ellipsoid with semi-axes (a, b, c) along
    (e1, e2, e3) centred in an n^3 periodic box and rotated about e1 by alpha (right-handed:
    its e3 axis turns towards -e2); a voxel is solid when its centre lies inside."""
    x = np.arange(n) + 0.5 - n / 2.0
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    t = np.radians(alpha_deg)
    yb = np.cos(t) * y + np.sin(t) * z   # body coordinates (rotation by -alpha)
    zb = -np.sin(t) * y + np.cos(t) * z
    a, b, c = semi
    return ((xx / a) ** 2 + (yb / b) ** 2 + (zb / c) ** 2 <= 1.0).astype(np.uint8)


def cylinder_cell(n: int, radius: float, ny: int, frame: int = 0) -> np.ndarray:
    """Regular thin porous medium of Sec. 6 ("2D microfluidic" unit cell): one solid
    cylinder of ``radius`` voxels with its axis along e2, centred in an n x n (e1, e3) cell,
    ``ny`` voxels thick along e2, the outer ``frame`` layers at both e2 ends solid.  Shape
    [n][ny][n] (z = e3, y = e2, x = e1)."""
    x = np.arange(n) + 0.5 - n / 2.0
    disk = (x[:, None] ** 2 + x[None, :] ** 2 <= radius * radius)  # [z][x]
    m = np.broadcast_to(disk[:, None, :], (n, ny, n)).astype(np.uint8).copy()
    if frame > 0:
        m[:, :frame, :] = 1
        m[:, ny - frame:, :] = 1
    return m


_LATTICE = {
    "sc": [(0.0, 0.0, 0.0)],
    "bcc": [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)],
    "fcc": [(0.0, 0.0, 0.0), (0.5, 0.5, 0.0), (0.5, 0.0, 0.5), (0.0, 0.5, 0.5)],
}


def regular_pack(L: int, kind: str, target_porosity: float):
    """Regular sphere packing of Sec. 6 in a periodic cubic unit cell of L voxels: spheres of
    one radius on the simple-cubic, body-centred or face-centred lattice sites (overlapping
    below the touching porosity).  The radius is the quantile of the distance of voxel
    centres to the nearest site at which the voxel porosity (centres inside a sphere are
    solid) reaches the target; voxels at equal distance go together, so small cells land
    within a per cent or two of it.  Returns (mask, radius in voxels)."""
    x = np.arange(L) + 0.5
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    d2 = np.full((L, L, L), np.inf)
    for (sx, sy, sz) in _LATTICE[kind]:
        dx = np.abs(xx - sx * L); dx = np.minimum(dx, L - dx)
        dy = np.abs(y - sy * L); dy = np.minimum(dy, L - dy)
        dz = np.abs(z - sz * L); dz = np.minimum(dz, L - dz)
        d2 = np.minimum(d2, dx * dx + dy * dy + dz * dz)
    d = np.sqrt(d2).ravel()
    n_solid = int(round((1.0 - target_porosity) * d.size))
    r = float(np.sort(d)[n_solid - 1]) if n_solid > 0 else 0.0
    return (np.sqrt(d2) <= r).astype(np.uint8), r


def random_blocks(shape, solid_fraction: float, seed: int) -> np.ndarray:
    """Independent random voxels, solid with probability ``solid_fraction``."""
    g = rng(seed)
    return (g.random(shape) < solid_fraction).astype(np.uint8)


def _paint_segment(dist: np.ndarray, a, b) -> None:
    """dist = min(dist, distance from voxel centres to segment a-b), periodic,
    evaluated in the bounding box of the segment grown by 4 voxels."""
    nz, ny, nx = dist.shape
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    lo = np.minimum(a, b) - 4.0
    hi = np.maximum(a, b) + 4.0
    axes = []
    for k, n in enumerate((nx, ny, nz)):
        idx = np.arange(int(np.floor(lo[k] - 0.5)), int(np.ceil(hi[k] - 0.5)) + 1)
        axes.append(idx)
    X, Y, Z = np.meshgrid(axes[0] + 0.5, axes[1] + 0.5, axes[2] + 0.5, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1)
    ab = b - a
    L2 = float(ab @ ab)
    t = np.clip(((P - a) @ ab) / L2, 0.0, 1.0) if L2 > 0 else np.zeros(P.shape[:-1])
    Q = a + t[..., None] * ab
    d = np.sqrt(np.sum((P - Q) ** 2, axis=-1))  # [x, y, z]
    ix = np.mod(axes[0], nx)
    iy = np.mod(axes[1], ny)
    iz = np.mod(axes[2], nz)
    sub = dist[np.ix_(iz, iy, ix)]
    np.minimum(sub, np.transpose(d, (2, 1, 0)), out=sub)
    dist[np.ix_(iz, iy, ix)] = sub


def voronoi_foam(n: int, n_seeds: int, strut_radius: float, target_porosity: float | None,
                 seed: int, tol: float = 0.02):
    """Open-cell foam: solid = voxels within ``strut_radius`` of an edge of the periodic
    Voronoi tessellation of ``n_seeds`` uniform seeds in an n^3 box.  If the porosity
    falls outside target +- tol, the radius is bisected to hit the target (the radius
    used is returned in info)."""
    from scipy.spatial import Voronoi

    g = rng(seed)
    pts = g.random((n_seeds, 3)) * n
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)],
                      dtype=np.float64) * n
    allp = np.concatenate([pts + s for s in shifts])
    vor = Voronoi(allp)
    edges = set()
    for rv in vor.ridge_vertices:
        if -1 in rv:
            continue
        for a, b in zip(rv, rv[1:] + rv[:1]):
            edges.add((min(a, b), max(a, b)))
    V = vor.vertices
    segs = []
    for a, b in edges:
        pa, pb = V[a], V[b]
        mid = 0.5 * (pa + pb)
        # keep each periodic edge once: the copy whose midpoint lies in [0, n)^3
        if np.all(mid >= 0) and np.all(mid < n):
            segs.append((pa, pb))
    dist = np.full((n, n, n), np.inf)
    for pa, pb in segs:
        _paint_segment(dist, pa, pb)
    r = strut_radius
    mask = (dist <= r).astype(np.uint8)
    if target_porosity is not None and abs(porosity(mask) - target_porosity) > tol:
        lo, hi = 0.5, 3.9
        for _ in range(40):
            r = 0.5 * (lo + hi)
            phi = float(np.count_nonzero(dist > r)) / dist.size
            if phi > target_porosity:
                lo = r
            else:
                hi = r
        mask = (dist <= r).astype(np.uint8)
    return mask, {"strut_radius": float(r), "n_edges": len(segs)}


def disk_cell(nx: int, ny: int, r_lo: float, r_hi: float, target_porosity: float, seed: int,
              max_rejections: int = 20000) -> np.ndarray:
    """2D periodic image [ny][nx] of non-overlapping disks, radii U[r_lo, r_hi],
    random sequential addition until the porosity reaches the target (or
    ``max_rejections`` consecutive rejections)."""
    g = rng(seed)
    box = np.array([nx, ny], dtype=np.float64)
    img = np.zeros((ny, nx), dtype=np.uint8)
    cs = np.zeros((0, 2))
    rs = np.zeros(0)
    rej = 0
    yy = np.arange(ny) + 0.5
    xx = np.arange(nx) + 0.5
    while rej < max_rejections and 1.0 - img.mean() > target_porosity:
        r = r_lo + (r_hi - r_lo) * g.random()
        c = g.random(2) * box
        if len(rs):
            d = cs - c
            d -= box * np.round(d / box)
            if not np.all(np.einsum("ij,ij->i", d, d) >= (rs + r) ** 2):
                rej += 1
                continue
        rej = 0
        cs = np.vstack([cs, c])
        rs = np.append(rs, r)
        dx = xx - c[0]
        dx -= nx * np.round(dx / nx)
        dy = yy - c[1]
        dy -= ny * np.round(dy / ny)
        img |= ((dy[:, None] ** 2 + dx[None, :] ** 2) <= r * r).astype(np.uint8)
    return img


def _extrude(img: np.ndarray, nz_fluid: int = 4) -> np.ndarray:
    """Quasi-2D cell: one solid layer, ``nz_fluid`` copies of the image, one solid layer."""
    ny, nx = img.shape
    m = np.ones((nz_fluid + 2, ny, nx), dtype=np.uint8)
    m[1:1 + nz_fluid] = img[None]
    return m


def clogging_sequence(nx: int = 1536, ny: int = 768, n_states: int = 24, phi0: float = 0.55,
                      phi_end: float = 0.30, seed: int = 3, nz_fluid: int = 4, r_lo: float = 12.0,
                      r_hi: float = 30.0):
    """Precipitation stand-in: a disk image (radii U[r_lo, r_hi]) at porosity phi0, then
    ``n_states`` states whose porosities fall linearly to phi_end by Eden growth (a random
    pore pixel with a solid 4-neighbour turns solid), identical in every fluid layer."""
    img = disk_cell(nx, ny, r_lo, r_hi, phi0, seed)
    states = []
    cur = img.copy()
    for s in range(n_states):
        phi_s = phi0 - s * (phi0 - phi_end) / max(n_states - 1, 1)
        g = rng(seed + s)
        target_solid = int(round((1.0 - phi_s) * cur.size))
        while np.count_nonzero(cur) < target_solid:
            nb = (np.roll(cur, 1, 0) | np.roll(cur, -1, 0) | np.roll(cur, 1, 1) | np.roll(cur, -1, 1))
            front = np.flatnonzero((cur == 0) & (nb == 1))
            need = target_solid - int(np.count_nonzero(cur))
            take = g.choice(front, size=min(need, max(1, len(front) // 8)), replace=False)
            cur.flat[take] = 1
        states.append(_extrude(cur, nz_fluid))
    return states


def crops(states, n_crops: int = 8, lo: int = 256, hi: int = 1024, seed: int = 100, multiple: int = 1):
    """Sub-domains of uneven in-plane sizes cut from randomly chosen states; the sizes are
    drawn uniformly in [lo, hi] (capped by the image) and rounded down to a multiple of
    ``multiple`` voxels (1: any size)."""
    g = rng(seed)
    out = []
    for _ in range(n_crops):
        st = states[int(g.integers(len(states)))]
        nz, ny, nx = st.shape
        cx = int(g.integers(lo, min(hi, nx) + 1)) // multiple * multiple
        cy = int(g.integers(lo, min(hi, ny) + 1)) // multiple * multiple
        ox = int(g.integers(0, nx - cx + 1))
        oy = int(g.integers(0, ny - cy + 1))
        out.append(np.ascontiguousarray(st[:, oy:oy + cy, ox:ox + cx]))
    return out


def boolean_spheres_gpu(n: int, r_lo: float, r_hi: float, target_porosity: float, seed: int,
                        device="cuda", chunk: int = 256):
    """Large periodic Boolean model (overlapping spheres, radii U[r_lo, r_hi]) on an n^3
    grid, rasterised on the GPU with torch.  The number of spheres is fixed in advance
    from the Boolean-model relation  porosity = exp(-density * E[sphere volume]), so the
    porosity is target_porosity up to sampling noise (the achieved value is returned).
    Centres and radii come from the seeded NumPy stream.  Returns (torch uint8 mask on
    ``device``, info)."""
    import torch

    g = rng(seed)
    ev = 4.0 / 3.0 * np.pi * (r_hi**4 - r_lo**4) / (4.0 * (r_hi - r_lo))  # E[r^3] for uniform r
    count = int(round(-np.log(target_porosity) * float(n) ** 3 / ev))
    centres = g.random((count, 3)) * n
    radii = r_lo + (r_hi - r_lo) * g.random(count)
    mask = torch.zeros((n, n, n), dtype=torch.uint8, device=device)
    R = int(np.ceil(r_hi)) + 1
    off = torch.arange(-R, R + 1, device=device, dtype=torch.float64)
    for s in range(0, count, chunk):
        c = torch.as_tensor(centres[s:s + chunk], device=device)
        r = torch.as_tensor(radii[s:s + chunk], device=device)
        base = torch.floor(c - 0.5)  # voxel whose centre is just below the centre
        # candidate voxel indices per axis: base + off; centre distance (idx + 1/2 - c)
        ix = base[:, None, :] + off[None, :, None]          # [k, 2R+1, 3]
        dd = ix + 0.5 - c[:, None, :]
        d2 = dd[:, :, None, None, 2] ** 2 + dd[:, None, :, None, 1] ** 2 + dd[:, None, None, :, 0] ** 2
        inside = d2 <= (r * r)[:, None, None, None]
        k, a, b, cc = torch.nonzero(inside, as_tuple=True)
        iz = torch.remainder(ix[k, a, 2], n).long()
        iy = torch.remainder(ix[k, b, 1], n).long()
        ixx = torch.remainder(ix[k, cc, 0], n).long()
        mask[iz, iy, ixx] = 1
    phi = 1.0 - float(mask.float().mean())
    return mask, {"spheres": count, "porosity": phi}
