"""Seeded synthetic inputs: Kuhn meshes of a cuboid, layered materials, pulse
centres and source positions.

This module only builds inputs (vertex coordinates, cell-to-vertex lists, cell
materials, random positions).  It holds none of the solver's arithmetic and
is the only code shared by the tests of the CUDA path and of the CPU checker.

Mesh recipe: n_x * n_y * n_z hexahedra on [-Lx,Lx] x [-Ly,Ly] x [-Lz,Lz],
each split into the 6 Kuhn (Freudenthal) tetrahedra along its (0,0,0)-(1,1,1)
diagonal, which is conforming because every hexahedron uses the same
diagonal.  Vertices are jittered uniformly by up to +/- jitter * h per
coordinate: interior vertices in 3D, face vertices tangentially, edge vertices
along the edge, corners fixed.  The jitter of a vertex depends only on
(seed, integer vertex position relative to the domain centre, axis), through
the splitmix64 counter-based generator, so nested domains share the jitter of
their common interior vertices.
"""
import itertools

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x):
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
    x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
    x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
    return x ^ (x >> np.uint64(31))


def hashed_uniform(seed, *ints):
    """Uniform [0,1) numbers keyed by (seed, i0, i1, ...) (broadcast arrays)."""
    with np.errstate(over="ignore"):
        h = _splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * np.ones(1, np.uint64))
        for v in ints:
            v = np.asarray(v).astype(np.int64).astype(np.uint64)
            h = _splitmix64(h ^ v)
    return (h >> np.uint64(11)).astype(np.float64) / float(1 << 53)


def kuhn_mesh(n, half_width=1.0, jitter=0.0, seed=0):
    """Return (VX [Nv,3] float64, EToV [K,4] int32) for an n^3 (or (nx,ny,nz))
    Kuhn mesh of the box [-L, L]^3 (L may be a 3-vector)."""
    n = np.broadcast_to(np.asarray(n, dtype=np.int64), (3,))
    L = np.broadcast_to(np.asarray(half_width, dtype=np.float64), (3,))
    h = 2.0 * L / n
    I, J, Kk = np.meshgrid(np.arange(n[0] + 1), np.arange(n[1] + 1), np.arange(n[2] + 1), indexing="ij")
    idx = np.stack([I.ravel(order="F"), J.ravel(order="F"), Kk.ravel(order="F")], axis=1)  # x fastest
    VX = -L + idx * h
    if jitter > 0.0:
        for a in range(3):
            movable = (idx[:, a] > 0) & (idx[:, a] < n[a])
            rel = 2 * idx - n                     # integer position relative to the centre
            u = hashed_uniform(seed, rel[:, 0], rel[:, 1], rel[:, 2], np.full(len(idx), a))
            VX[movable, a] += (2.0 * u[movable] - 1.0) * jitter * h[a]
    nx1, ny1 = n[0] + 1, n[1] + 1

    def vid(i, j, k):
        return i + nx1 * (j + ny1 * k)

    hi, hj, hk = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    hi, hj, hk = hi.ravel(order="F"), hj.ravel(order="F"), hk.ravel(order="F")
    tets = []
    for perm in itertools.permutations(range(3)):
        path = [np.zeros(3, int)]
        for ax in perm:
            step = path[-1].copy()
            step[ax] += 1
            path.append(step)
        tets.append(np.stack([vid(hi + p[0], hj + p[1], hk + p[2]) for p in path], axis=1))
    EToV = np.stack(tets, axis=1).reshape(-1, 4)         # the 6 tets of a hex are consecutive
    # positive orientation: swap the last two vertices of negatively oriented tets
    v = VX[EToV]
    det = np.einsum("ki,ki->k", v[:, 1] - v[:, 0], np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))
    neg = det < 0
    EToV[neg, 2], EToV[neg, 3] = EToV[neg, 3].copy(), EToV[neg, 2].copy()
    return VX, EToV.astype(np.int32)


def layered_material(VX, EToV, z_tops, c_layers, rho_layers, hex_centroid=True):
    """Per-tet (c, rho) of horizontal layers listed bottom to top; layer l holds
    z < z_tops[l] (the last layer takes the rest).  With hex_centroid the six
    Kuhn tets of a hexahedron share the layer of the hexahedron centroid."""
    zc = VX[EToV].mean(axis=1)[:, 2]
    if hex_centroid and EToV.shape[0] % 6 == 0:
        zc = zc.reshape(-1, 6).mean(axis=1).repeat(6)
    layer = np.searchsorted(np.asarray(z_tops, float), zc, side="right")
    layer = np.minimum(layer, len(c_layers) - 1)
    return np.asarray(c_layers, float)[layer], np.asarray(rho_layers, float)[layer]


def seeded_point(seed, centre, spread):
    """centre + U(-spread, spread)^3 from the counter-based generator."""
    u = hashed_uniform(seed, np.arange(3), np.full(3, 7))
    return np.asarray(centre, float) + (2.0 * u - 1.0) * spread


def random_state(seed, shape, scale=1.0):
    """Reproducible uniform(-scale, scale) array of the given shape."""
    rng = np.random.Generator(np.random.Philox(seed))
    return (2.0 * rng.random(shape) - 1.0) * scale


def batch_problems(seed, count=48, n_range=(8, 24), orders=(3, 4, 5), habc_orders=(2, 4, 6), f_range=(2.0, 6.0),
                   src_box=0.5):
    """A seeded list of independent problems for the batching form: problem i
    has n ~ U{n_range} hexes per axis on [-1,1]^3 (jitter 2% h, mesh seed
    seed + i), degree N and HABC order P drawn uniformly from the given sets,
    c = rho = 1, and a Ricker point source of peak frequency f0 ~ U[f_range]
    at xs ~ U[-src_box, src_box]^3 with delay t_s = 1.25 / f0."""
    out = []
    for i in range(count):
        u = [float(hashed_uniform(seed, i, j)[0]) for j in range(7)]
        n = n_range[0] + int(u[0] * (n_range[1] - n_range[0] + 1))
        N = orders[int(u[1] * len(orders))]
        P = habc_orders[int(u[2] * len(habc_orders))]
        f0 = f_range[0] + u[3] * (f_range[1] - f_range[0])
        xs = [(2.0 * u[4 + a] - 1.0) * src_box for a in range(3)]
        out.append({"n": n, "N": N, "P": P, "f0": f0, "xs": xs, "t_s": 1.25 / f0, "mesh_seed": seed + i})
    return out


SEAM_DIMS = (56, 64, 24)
SEAM_HALF = (1.75, 2.0, 0.75)


def seam_standin(seed=7000):
    """The heterogeneous stand-in for the paper's SEAM setting (Sec. 4.2):
    box [-1.75,1.75] x [-2,2] x [-0.75,0.75], 56 x 64 x 24 hexahedra x 6 Kuhn
    tets (jitter 2% h); three horizontal layers by tet centroid, (c, rho) =
    (3.5, 2.4) for z < -0.25, (2.5, 2.1) for z < 0.25, (1.5, 1.8) above; a fast
    inclusion (4.5, 2.6) where x > 1.0, |y| < 0.5, -0.4 < z < 0.1 (it touches
    the +x face).  Returns (VX, EToV, c, rho)."""
    VX, EToV = kuhn_mesh(SEAM_DIMS, SEAM_HALF, 0.02, seed=seed)
    cen = VX[EToV].mean(axis=1)
    z = cen[:, 2]
    c = np.where(z < -0.25, 3.5, np.where(z < 0.25, 2.5, 1.5))
    rho = np.where(z < -0.25, 2.4, np.where(z < 0.25, 2.1, 1.8))
    inc = (cen[:, 0] > 1.0) & (np.abs(cen[:, 1]) < 0.5) & (z > -0.4) & (z < 0.1)
    c[inc], rho[inc] = 4.5, 2.6
    return VX, EToV, c, rho
