"""Seeded synthetic inputs for the unstructured S_N sweep.

This module only draws random numbers and lays out input arrays: it holds none
of the transport method's arithmetic (no geometry, no quadrature, no sweep).
Both the CUDA library's tests/bench and the CPU oracle consume what it returns.

Random numbers: SplitMix64 in counter form.  Output i (i = 0, 1, ...) of a stream
with seed s is mix(s + (i+1)*0x9E3779B97F4A7C15) where mix is the SplitMix64
finaliser (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
0x94D049BB133111EB, xor-shift 31).  A uniform double is (x >> 11) * 2**-53.
Each purpose (jitter, materials, cross sections, sources, batch sizes) draws
from its own stream whose seed is base_seed + purpose * 2**32.

Mesh recipe (jittered hex box, Kuhn split):
  * vertices (i, j, k) * h, h = 1/n, index v = i + (n+1)*(j + (n+1)*k);
  * interior vertices (0 < i, j, k < n) move by (2u - 1) * jitter * h in each
    coordinate d, u = output 3*v + d of the jitter stream (boundary draws unused);
  * hex (i, j, k), id i + n*(j + n*k), splits into 6 tetrahedra, one per axis
    permutation p in the order xyz, xzy, yxz, yzx, zxy, zyx: the tet walks from
    vertex (i, j, k) by unit steps along p[0], p[1], p[2]; for odd permutations
    local vertices 2 and 3 are swapped so that every tet is positively oriented
    (the determinant of the unjittered walk equals the permutation's sign);
  * cell id = 6 * hex id + p.

The paper measures on UnSNAP's synthetic twisted-hex grids; the configurations
below are seeded stand-ins with the shapes of that workload (S_N directions,
energy groups, material blocks, box sources) on tetrahedra.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

# purposes: one independent stream each
P_JITTER, P_MATERIAL, P_XS, P_SOURCE, P_BATCH, P_LAYOUT = range(6)

BASE_SEED = 2510115130

PERMUTATIONS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
ODD_PERMUTATION = (False, True, True, False, False, True)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the counter-form SplitMix64 stream `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + i * GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): (x >> 11) * 2**-53."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def stream_seed(base: int, purpose: int) -> int:
    return (base + purpose * (1 << 32)) % (1 << 64)


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def uniform(self, n: int) -> np.ndarray:
        u = uniform(self.seed, n, self.pos)
        self.pos += n
        return u


# --------------------------------------------------------------------------- mesh
def jittered_kuhn_mesh(n: int, seed: int, jitter: float = 0.15):
    """Jittered n^3 hex box on [0,1]^3, each hex Kuhn-split into 6 tets.

    Returns (xyz [(n+1)^3, 3] float64, tets [6 n^3, 4] int32).
    """
    n1 = n + 1
    h = 1.0 / n
    k, j, i = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)  # row v = i + n1*(j + n1*k)
    xyz = ijk.astype(np.float64) * h
    if jitter != 0.0 and n > 1:
        u = uniform(stream_seed(seed, P_JITTER), 3 * n1 ** 3).reshape(-1, 3)
        interior = np.all((ijk > 0) & (ijk < n), axis=1)
        xyz[interior] += (2.0 * u[interior] - 1.0) * (jitter * h)
    hk, hj, hi = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()  # hex id = hi + n*(hj + n*hk)
    steps = np.array([1, n1, n1 * n1], dtype=np.int64)  # vertex-index step along x, y, z
    v0 = hi + n1 * (hj + n1 * hk)
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for p, perm in enumerate(PERMUTATIONS):
        a = v0
        b = a + steps[perm[0]]
        c = b + steps[perm[1]]
        d = c + steps[perm[2]]
        if ODD_PERMUTATION[p]:
            c, d = d, c
        tets[:, p] = np.stack([a, b, c, d], axis=1)
    return xyz, tets.reshape(-1, 4).astype(np.int32)


def hex_index_of_cells(n: int) -> np.ndarray:
    """(i, j, k) of the parent hex of every cell, shape [6 n^3, 3]."""
    h = np.arange(n ** 3)
    ijk = np.stack([h % n, (h // n) % n, h // (n * n)], axis=1)
    return np.repeat(ijk, 6, axis=0)


# ------------------------------------------------------------------ cross sections
def downscatter_matrix(sig_t: np.ndarray, ratio: np.ndarray, st: Stream, upscatter: float = 0.0):
    """Scattering matrix [g_from][g_to] for one material.

    Row g (the from-group) sums to ratio[g] * sig_t[g].  A fraction `upscatter`
    of it is spread evenly over g' < g (group 0 gets none: its whole row goes
    down); the rest is split over g' >= g with U(0,1) weights normalised to 1.
    Draw order: for g = 0..G-1, (G - g) weights.
    """
    G = sig_t.shape[0]
    S = np.zeros((G, G))
    for g in range(G):
        total = ratio[g] * sig_t[g]
        wts = st.uniform(G - g)
        wts = wts / wts.sum() if wts.sum() > 0 else np.full(G - g, 1.0 / (G - g))
        up = upscatter if g > 0 else 0.0
        S[g, g:] = (1.0 - up) * total * wts
        if g > 0 and up > 0.0:
            S[g, :g] = up * total / g
    return S


def _log_uniform(u, lo, hi):
    return lo * (hi / lo) ** u


# ------------------------------------------------------------------ configurations
def _problem(n, seed, n_polar, n_az, G, M, cell_material, sigma_t, sigma_s, Q, tol, precision, name):
    xyz, tets = jittered_kuhn_mesh(n, seed)
    return dict(
        name=name, n=n, seed=seed, xyz=xyz, tets=tets, n_polar=n_polar, n_azimuthal=n_az,
        n_groups=G, n_materials=M, cell_material=np.ascontiguousarray(cell_material, dtype=np.int32),
        sigma_t=np.ascontiguousarray(sigma_t, dtype=np.float64),
        sigma_s=np.ascontiguousarray(sigma_s, dtype=np.float64),
        Q=np.ascontiguousarray(Q, dtype=np.float64), tol=tol, precision=precision,
    )


def small_box(n=8, G=4, n_polar=4, n_az=8, seed=BASE_SEED + 1, tol=1e-8, precision="f64"):
    """One material, sigma_t ~ U[0.5, 2], downscatter rows summing to 0.5 sigma_t,
    Q = 1 in the central hexes (the hexes inside [0.375, 0.625]^3 when n = 8).

    Draw order (cross-section stream): G values for sigma_t, then the
    downscatter weights.
    """
    C = 6 * n ** 3
    st = Stream(stream_seed(seed, P_XS))
    sig_t = 0.5 + 1.5 * st.uniform(G)
    S = downscatter_matrix(sig_t, np.full(G, 0.5), st)
    hx = hex_index_of_cells(n)
    lo, hi = (3 * n) // 8, (5 * n) // 8  # hexes [3,4] of 8 => [0.375, 0.625]
    src = np.all((hx >= lo) & (hx < hi), axis=1)
    Q = np.zeros((C, G, 4))
    Q[src] = 1.0
    return _problem(n, seed, n_polar, n_az, G, 1, np.zeros(C), sig_t[None, :], S[None], Q, tol,
                    precision, f"small_box_{n}^3_D{n_polar * n_az}_G{G}")


def block_materials(n, block, M, st: Stream):
    """Material per cell from random block x block x block hex blocks (one draw per block)."""
    nb = -(-n // block)
    u = st.uniform(nb ** 3)
    mat_of_block = np.minimum((u * M).astype(np.int64), M - 1)
    hx = hex_index_of_cells(n) // block
    return mat_of_block[hx[:, 0] + nb * (hx[:, 1] + nb * hx[:, 2])]


def material_xs(M, G, st: Stream, c_lo, c_hi, upscatter):
    """Per material: sigma_t log-uniform in [0.1, 10] (G draws), scattering ratio
    c ~ U[c_lo, c_hi] (G draws), then the scattering weights."""
    sig_t = np.zeros((M, G))
    S = np.zeros((M, G, G))
    for m in range(M):
        sig_t[m] = _log_uniform(st.uniform(G), 0.1, 10.0)
        ratio = c_lo + (c_hi - c_lo) * st.uniform(G)
        S[m] = downscatter_matrix(sig_t[m], ratio, st, upscatter)
    return sig_t, S


def two_material_box(n=32, G=32, n_polar=8, n_az=16, seed=BASE_SEED + 2, tol=1e-6, precision="f32"):
    """Two materials on random 4x4x4-hex blocks, sigma_t log-uniform [0.1, 10],
    c ~ U[0.3, 0.9], downscatter plus 5 % upscatter, Q = 1 in the first material."""
    C = 6 * n ** 3
    mat = block_materials(n, 4, 2, Stream(stream_seed(seed, P_MATERIAL)))
    sig_t, S = material_xs(2, G, Stream(stream_seed(seed, P_XS)), 0.3, 0.9, 0.05)
    Q = np.zeros((C, G, 4))
    Q[mat == 0] = 1.0
    return _problem(n, seed, n_polar, n_az, G, 2, mat, sig_t, S, Q, tol, precision,
                    f"two_material_{n}^3_D{n_polar * n_az}_G{G}")


def corner_source_box(n=48, G=64, n_polar=12, n_az=16, seed=BASE_SEED + 3, tol=1e-6, precision="f32"):
    """Four materials on random 6x6x6-hex blocks, sigma_t log-uniform [0.1, 10],
    c ~ U[0.5, 0.95], downscatter only, Q = 1 in the corner hex (0, 0, 0)."""
    C = 6 * n ** 3
    mat = block_materials(n, max(1, n // 8), 4, Stream(stream_seed(seed, P_MATERIAL)))
    sig_t, S = material_xs(4, G, Stream(stream_seed(seed, P_XS)), 0.5, 0.95, 0.0)
    Q = np.zeros((C, G, 4))
    Q[:6] = 1.0
    return _problem(n, seed, n_polar, n_az, G, 4, mat, sig_t, S, Q, tol, precision,
                    f"corner_source_{n}^3_D{n_polar * n_az}_G{G}")


def batch_of_problems(count=64, seed=BASE_SEED + 4, n_range=(12, 40), tol=1e-6, precision="f32"):
    """Independent problems of uneven size: n ~ U{n_range}, D in {32, 64, 128}
    (4x8, 8x8, 8x16), G in {8, 16, 32, 64}; materials and cross sections as in
    two_material_box.  Draw order (batch stream): per problem n, D choice, G choice."""
    st = Stream(stream_seed(seed, P_BATCH))
    dirs = ((4, 8), (8, 8), (8, 16))
    groups = (8, 16, 32, 64)
    out = []
    for p in range(count):
        u = st.uniform(3)
        n = n_range[0] + min(int(u[0] * (n_range[1] - n_range[0] + 1)), n_range[1] - n_range[0])
        npol, naz = dirs[min(int(u[1] * 3), 2)]
        G = groups[min(int(u[2] * 4), 3)]
        out.append(two_material_box(n=n, G=G, n_polar=npol, n_az=naz, seed=seed + 1000 * (p + 1),
                                    tol=tol, precision=precision))
    return out


def random_layout(n=24, G=16, n_polar=8, n_az=8, seed=BASE_SEED + 5, layout=0, tol=1e-6, precision="f32"):
    """Learned-start layouts: sigma_t log-uniform [0.1, 10] per (3x3x3-hex block,
    group), scattering ratio c ~ U[0.3, 0.99] per block (downscatter only), one
    to three random hex-aligned box sources with Q ~ U[0, 1].  Each block is its
    own material.  Layout k uses seed + 7919 * k."""
    s = seed + 7919 * layout
    C = 6 * n ** 3
    blk = 3
    nb = -(-n // blk)
    M = nb ** 3
    hx = hex_index_of_cells(n)
    b = hx // blk
    mat = b[:, 0] + nb * (b[:, 1] + nb * b[:, 2])
    sig_t, S = material_xs(M, G, Stream(stream_seed(s, P_XS)), 0.3, 0.99, 0.0)
    st = Stream(stream_seed(s, P_SOURCE))
    nbox = 1 + min(int(st.uniform(1)[0] * 3), 2)
    Q = np.zeros((C, G, 4))
    for _ in range(nbox):
        u = st.uniform(6 + G)
        lo = np.minimum((u[0:3] * n).astype(int), n - 1)
        ext = 1 + (u[3:6] * (n // 4)).astype(int)
        hi = np.minimum(lo + ext, n)
        inside = np.all((hx >= lo) & (hx < hi), axis=1)
        Q[inside] += u[6:6 + G][None, :, None]
    return _problem(n, s, n_polar, n_az, G, M, mat, sig_t, S, Q, tol, precision,
                    f"layout{layout}_{n}^3_D{n_polar * n_az}_G{G}")


def paper_context_box(n=16, G=16, n_polar=8, n_az=16, seed=BASE_SEED + 6):
    """16^3 hexes, 128 directions, 16 groups: the size of the paper's runtime table
    workload (hexes there, Kuhn tets here), one material as small_box."""
    p = small_box(n=n, G=G, n_polar=n_polar, n_az=n_az, seed=seed, tol=1e-6, precision="f32")
    p["name"] = f"paper_context_{n}^3_D{n_polar * n_az}_G{G}"
    return p


def order2(cfg):
    """The same problem for the second-order (ten-node) element: Q at the four
    vertices and, at the six edge midpoints (0,1) (0,2) (0,3) (1,2) (1,3) (2,3),
    the mean of the edge's two vertex values (the same linear field per cell)."""
    Q = np.asarray(cfg["Q"], dtype=np.float64)
    mids = [0.5 * (Q[..., a] + Q[..., b]) for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))]
    out = dict(cfg)
    out["Q"] = np.concatenate([Q, np.stack(mids, axis=-1)], axis=-1)
    out["order"] = 2
    out["name"] = cfg.get("name", "") + "_P2"
    return out


def order3(cfg):
    """The same problem for the third-order (twenty-node) element: Q at the vertices,
    at the two nodes of each edge (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) (at 1/3 and 2/3
    from the edge's first vertex) and at the four face centres, each the value of the
    cell's linear field through its four vertex values."""
    Q = np.asarray(cfg["Q"], dtype=np.float64)
    bary = [tuple(1.0 if k == v else 0.0 for k in range(4)) for v in range(4)]
    for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)):
        for t in (2.0 / 3.0, 1.0 / 3.0):
            bary.append(tuple(t if k == a else (1.0 - t if k == b else 0.0) for k in range(4)))
    for f in range(4):
        bary.append(tuple(0.0 if k == f else 1.0 / 3.0 for k in range(4)))
    out = dict(cfg)
    out["Q"] = np.einsum("cgk,ik->cgi", Q, np.array(bary))
    out["order"] = 3
    out["name"] = cfg.get("name", "") + "_P3"
    return out


def paper_hex_box(n=16, G=10, n_polar=8, n_az=32, seed=BASE_SEED + 7, twist=0.25):
    """The paper's runtime-table workload as far as it is stated: 16^3 trilinear hexahedra
    (the orthogonal grid twisted along one axis), 10 energy groups, 32 directions per octant
    (8 polar x 32 azimuthal = 256); one material and the central box source as small_box."""
    p = hex_problem(small_box(n=n, G=G, n_polar=n_polar, n_az=n_az, seed=seed, tol=1e-6, precision="f32"),
                    twist=twist)
    p["name"] = f"paper_hex_{n}^3_D{n_polar * n_az}_G{G}_twist{twist:g}"
    return p


CONFIGS = {
    "small_box": small_box,
    "two_material": two_material_box,
    "corner_source": corner_source_box,
    "batch": batch_of_problems,
    "layout": random_layout,
    "paper_context": paper_context_box,
}  # the hexahedral workloads join below, after their generators


# ------------------------------------------------------------------ hexahedra
def twisted_hex_mesh(n: int, seed: int, jitter: float = 0.15, twist: float = 0.0):
    """The n^3 hex box of `jittered_kuhn_mesh` (the same vertices and jitter draws) kept as
    hexahedra and then twisted about the vertical line x = y = 1/2: a vertex at height z
    turns by twist * z radians in the horizontal plane (twist = 0: no turn).

    Returns (xyz [(n+1)^3, 3] float64, hexes [n^3, 8] int32).  Hex (i, j, k) has id
    i + n*(j + n*k); its local vertex a + 2b + 4c (a, b, c in {0, 1}) is mesh vertex
    (i + a, j + b, k + c).
    """
    xyz, _ = jittered_kuhn_mesh(n, seed, jitter)
    if twist != 0.0:
        t = twist * xyz[:, 2]
        ct, sn = np.cos(t), np.sin(t)
        x, y = xyz[:, 0] - 0.5, xyz[:, 1] - 0.5
        xyz[:, 0] = 0.5 + (ct * x - sn * y)
        xyz[:, 1] = 0.5 + (sn * x + ct * y)
    n1 = n + 1
    hk, hj, hi = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    v0 = (hi.ravel() + n1 * (hj.ravel() + n1 * hk.ravel())).astype(np.int64)
    hexes = np.empty((n ** 3, 8), dtype=np.int64)
    for v in range(8):
        a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
        hexes[:, v] = v0 + a + n1 * (b + n1 * c)
    return xyz, hexes.astype(np.int32)


def hex_problem(cfg, twist: float = 0.25, jitter: float = 0.0):
    """The same problem on trilinear hexahedra: the parent hexes of a tetrahedral
    configuration above (same material per hex, same cross sections) on the orthogonal
    n^3 grid twisted by `twist` radians over the box height (the paper's synthetic mesh
    kind; `jitter` > 0 moves interior vertices as for the tetrahedral meshes).  Q becomes
    [n^3][G][8]: every configuration here holds Q constant over a parent hex, and each
    hex takes the mean of its six tetrahedra's nodal values.

    Sweep graphs of twisted grids can hold cycles (a face's integrated normal decides its
    direction, and a non-planar face can tilt against its neighbours): with no jitter,
    twist 0.25 gave acyclic graphs for 32, 128 and 256 product directions on 8^3 and 16^3
    grids, twist 0.5 did not at 128 directions, and jitter 0.15 did not at 128."""
    n = int(cfg["n"])
    xyz, hexes = twisted_hex_mesh(n, int(cfg["seed"]), jitter=jitter, twist=twist)
    G = int(cfg["n_groups"])
    Qt = np.asarray(cfg["Q"], dtype=np.float64).reshape(n ** 3, 6, G, -1)
    Q = np.repeat(Qt.mean(axis=(1, 3))[:, :, None], 8, axis=2)
    out = dict(cfg)
    out.update(xyz=xyz, hexes=hexes, element="hex", twist=twist, jitter=jitter,
               cell_material=np.ascontiguousarray(np.asarray(cfg["cell_material"])[::6], dtype=np.int32),
               Q=np.ascontiguousarray(Q), name=cfg.get("name", "") + f"_hex_twist{twist:g}")
    out.pop("tets", None)
    return out


def two_material_hex(**kw):
    """The two-material box as a twisted hex grid (twist 0.25, no jitter)."""
    return hex_problem(two_material_box(**kw))


CONFIGS["paper_hex"] = paper_hex_box
CONFIGS["two_material_hex"] = two_material_hex
