"""Seeded synthetic inputs shaped like the paper's random suspensions.

This module only draws particle positions, forces and torques. It holds none of
the fast-FCM arithmetic, so both the CUDA path (through the tests and the bench)
and the CPU oracle (through the tests) can take their inputs from here.

Workloads follow the paper's experiments (Section 5: random, non-overlapping
suspensions of spheres of radius a in a periodic cube at volume fraction phi)
and the rod layouts of Section 6.1 (spheres stacked along rigid rods):

* ``random_suspension``: uniform random sequential addition (RSA) with a minimum
  centre separation (2.2a by default), box edge from N and phi.
* ``random_rods``: rods of ``per_rod`` spheres at a fixed bond spacing, centres
  uniform and axes isotropic, RSA at the sphere level.
* ``random_loads``: forces and torques i.i.d. N(0, 1) per component with the
  mean removed.
"""
from __future__ import annotations

import math

import numpy as np

try:  # neighbour queries for the rejection step only
    from scipy.spatial import cKDTree as _KDTree
except Exception:  # pragma: no cover - scipy is present on both machines
    _KDTree = None

#: base seed for every generated workload (paper id 2310.12651, then a digit)
BASE_SEED = 2310126510


def box_edge(n: int, phi: float, a: float = 1.0) -> float:
    """Edge L of the periodic cube holding n spheres of radius a at volume fraction phi."""
    return (n * 4.0 * math.pi * a ** 3 / (3.0 * phi)) ** (1.0 / 3.0)


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def random_suspension(n: int, L: float, seed: int, min_sep: float = 2.2,
                      max_rounds: int = 200) -> np.ndarray:
    """n points uniform in [0, L)^3 with periodic centre separation >= min_sep.

    Candidates are drawn in batches; a candidate is kept if it is at least
    ``min_sep`` from every kept point and from every earlier candidate kept in
    the same batch. Returns float64 (n, 3).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if n == 0:
        return np.zeros((0, 3))
    if min_sep <= 0:
        return rng.random((n, 3)) * L
    if _KDTree is None:
        raise RuntimeError("scipy is required for the rejection step")
    kept = np.zeros((0, 3))
    for _ in range(max_rounds):
        need = n - kept.shape[0]
        if need <= 0:
            break
        cand = rng.random((max(64, int(need * 1.3)), 3)) * L
        cand = np.minimum(cand, np.nextafter(L, 0))
        ok = np.ones(cand.shape[0], dtype=bool)
        if kept.shape[0]:
            tree = _KDTree(kept, boxsize=L)
            d, _ = tree.query(cand, k=1)
            ok &= d >= min_sep
        # resolve conflicts inside the batch: the lower index wins
        ctree = _KDTree(cand, boxsize=L)
        pairs = ctree.query_pairs(np.nextafter(min_sep, 0), output_type="ndarray")
        if pairs.size:
            order = np.argsort(pairs[:, 0], kind="stable")
            for i, j in pairs[order]:
                if ok[i] and ok[j]:
                    ok[j] = False
        kept = np.concatenate([kept, cand[ok][:need]], axis=0)
    if kept.shape[0] < n:
        raise RuntimeError(f"RSA placed only {kept.shape[0]} of {n} spheres")
    return kept


def random_rods(n_rods: int, per_rod: int, L: float, seed: int, bond: float = 2.2,
                min_sep: float = 2.2, max_attempts: int = 400000, stall: int = 300,
                cone_cos: float = 0.98) -> tuple[np.ndarray, float]:
    """Rigid rods of ``per_rod`` spheres spaced ``bond`` apart along a random axis.

    Rod centres are uniform in the box and axes uniform on the sphere. A rod is
    rejected if any of its spheres lies closer than ``min_sep`` to a sphere of an
    accepted rod (periodic distance). Long rods jam well below the isotropic-
    nematic density; after ``stall`` consecutive rejections the remaining rods
    are drawn with axes inside a cone around z (cos theta >= ``cone_cos``), which
    packs. Returns (positions wrapped into [0, L), the volume fraction reached
    with radius 1 spheres); ``random_rods.last_stats`` records how many rods were
    isotropic and how many aligned. ``min_sep <= 0`` skips the rejection (rods may
    cross), for workloads where only the layout's clustering matters.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    offs = (np.arange(per_rod) - 0.5 * (per_rod - 1)) * bond
    if min_sep <= 0:   # no rejection: rods may cross each other (spheres within a rod stay bond apart)
        c = rng.random((n_rods, 3)) * L
        v = rng.normal(size=(n_rods, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        pos = np.mod(c[:, None, :] + offs[None, :, None] * v[:, None, :], L).reshape(-1, 3)
        pos = np.minimum(pos, np.nextafter(L, 0))
        random_rods.last_stats = {"isotropic": n_rods, "aligned": 0, "attempts": n_rods}
        return pos, pos.shape[0] * 4.0 * math.pi / 3.0 / L ** 3
    accepted: list[np.ndarray] = []
    tree = None
    pending: list[np.ndarray] = []
    attempts = rejections = 0
    aligned = False
    n_iso = 0
    while len(accepted) < n_rods and attempts < max_attempts:
        attempts += 1
        c = rng.random(3) * L
        if aligned:
            cz = rng.uniform(cone_cos, 1.0)
            ph = rng.uniform(0.0, 2 * np.pi)
            sz = np.sqrt(1.0 - cz * cz)
            v = np.array([sz * np.cos(ph), sz * np.sin(ph), cz])
        else:
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
        pts = np.mod(c[None, :] + offs[:, None] * v[None, :], L)
        pts = np.minimum(pts, np.nextafter(L, 0))
        bad = False
        if tree is not None:
            d, _ = tree.query(pts, k=1)
            bad = bool(np.any(d < min_sep))
        if not bad and pending:
            q = np.concatenate(pending, axis=0)
            dd = _min_image(pts[:, None, :] - q[None, :, :], L)
            bad = bool(np.any(np.einsum("ijk,ijk->ij", dd, dd) < min_sep ** 2))
        if bad:
            rejections += 1
            if not aligned and rejections >= stall:
                aligned = True
            continue
        rejections = 0
        accepted.append(pts)
        if not aligned:
            n_iso += 1
        pending.append(pts)
        if len(pending) >= 16:
            tree = _KDTree(np.concatenate(accepted, axis=0), boxsize=L)
            pending = []
    random_rods.last_stats = {"isotropic": n_iso, "aligned": len(accepted) - n_iso, "attempts": attempts}
    if not accepted:
        return np.zeros((0, 3)), 0.0
    pos = np.concatenate(accepted, axis=0)
    phi = pos.shape[0] * 4.0 * math.pi / 3.0 / L ** 3
    return pos, phi


def random_loads(n: int, seed: int, torques: bool = True, mean_free: bool = True,
                 scale: float = 1.0, bias=None) -> tuple[np.ndarray, np.ndarray | None]:
    """Forces (and torques) i.i.d. N(0, scale^2) per component, optionally mean-free.

    ``bias`` (3-vector) is added to every force after the mean is removed, as
    for the sedimenting-rod layout (a constant gravity force per sphere).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    F = rng.normal(size=(n, 3)) * scale
    T = rng.normal(size=(n, 3)) * scale if torques else None
    if mean_free and n > 0:
        F -= F.mean(axis=0, keepdims=True)
        if T is not None:
            T -= T.mean(axis=0, keepdims=True)
    if bias is not None:
        F = F + np.asarray(bias, dtype=np.float64)[None, :]
    return F, T


#: FCM particles per rod and the doublet layout of the sedimenting-rod suspensions (Section 6.1)
ROD_DOUBLETS = 11
ROD_PITCH = math.sqrt(2.0)   # axial distance between consecutive doublets, in units of a


def doublet_rods(n_rods: int, L_xy: float, L_z: float, seed: int, doublets: int = ROD_DOUBLETS,
                 a: float = 1.0, lattice: bool = True) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Planar rods built from alternating doublets of FCM particles (Section 6.1).

    A rod has ``doublets`` doublets spaced ``ROD_PITCH * a`` along its axis; the two
    particles of a doublet sit at +-a from the axis, alternately along the in-plane
    normal and along z, so neighbouring particles are 2a apart and 11 doublets give
    the rod length 10 sqrt(2) a = 14.14a. Rod centres lie in the plane z = L_z/2 on a
    square lattice (``lattice``) or uniformly at random, axes in the plane at a random
    angle. Returns (positions wrapped into the box (n_rods * 2 * doublets, 3),
    body offsets (n_rods + 1,) int32, rod centres (n_rods, 3)); the particles of rod b
    are rows body_off[b] .. body_off[b+1]-1 and rod b's centre is their centroid.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    per = 2 * doublets
    if lattice:
        side = int(math.ceil(math.sqrt(n_rods)))
        spacing = L_xy / side
        k = np.arange(n_rods)
        cx = (k % side + 0.5) * spacing
        cy = (k // side + 0.5) * spacing
    else:
        cx = rng.random(n_rods) * L_xy
        cy = rng.random(n_rods) * L_xy
    centres = np.stack([cx, cy, np.full(n_rods, 0.5 * L_z)], axis=1)
    th = rng.uniform(0.0, 2.0 * math.pi, n_rods)
    axis = np.stack([np.cos(th), np.sin(th), np.zeros(n_rods)], axis=1)
    normal = np.stack([-np.sin(th), np.cos(th), np.zeros(n_rods)], axis=1)
    ez = np.array([0.0, 0.0, 1.0])
    off = np.empty((n_rods, per, 3))
    for d in range(doublets):
        s = (d - 0.5 * (doublets - 1)) * ROD_PITCH * a
        lat = normal if d % 2 == 0 else np.broadcast_to(ez, (n_rods, 3))
        off[:, 2 * d] = s * axis + a * lat
        off[:, 2 * d + 1] = s * axis - a * lat
    box = np.array([L_xy, L_xy, L_z])
    pos = np.mod(centres[:, None, :] + off, box).reshape(-1, 3)
    pos = np.minimum(pos, np.nextafter(box, 0))
    body_off = (np.arange(n_rods + 1) * per).astype(np.int32)
    return pos, body_off, centres


def rod_loads(n_rods: int, seed: int, gravity=(1.0, 0.0, 0.0), per_rod: int = 2 * ROD_DOUBLETS,
              scale: float = 0.0) -> np.ndarray:
    """Rod forces and torques (n_rods, 6): per_rod * gravity plus i.i.d. N(0, scale^2) parts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ft = rng.normal(size=(n_rods, 6)) * scale
    ft[:, :3] += per_rod * np.asarray(gravity, dtype=np.float64)[None, :]
    return ft
