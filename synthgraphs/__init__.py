"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module builds graphs (as CSR adjacency patterns) and start vectors. It
holds none of the eigensolver's arithmetic: no Laplacian, no operator, no
Krylov step. Everything it returns is *input data* for the graph Laplacian
eigenvalue problem L x = lambda x of a simple, connected, undirected,
unweighted graph (paper Sec. 1.1, Eq. 1.1, Theorem 1.2).

Randomness comes from one counter-based generator, SplitMix64 (S. Vigna,
"Further scramblings of Marsaglia's xorshift generators", public domain
definition): value(seed, c) is the SplitMix64 output after c+1 increments of
the golden-gamma counter started at `seed`.  It is implemented here with
numpy's wrapping uint64 arithmetic, so results are identical on every host.

CSR convention used everywhere in this project:
  row_ptr : int64[n+1], col_idx : int32[nnz], rows sorted ascending,
  symmetric pattern, no self loops, no duplicates, no values array
  (unit weights: the degree of row r is row_ptr[r+1]-row_ptr[r]).
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """SplitMix64 output number `counter` (0-based) of the stream started at `seed`."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64(seed, counter)."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def stream_seed(*parts: int) -> int:
    """Derive a 64-bit stream seed from a tuple of small integers (e.g. (seed, graph_index))."""
    s = 0x243F6A8885A308D3
    for p in parts:
        s = int(splitmix64(s ^ (int(p) & 0xFFFFFFFFFFFFFFFF), 0))
    return s


# --------------------------------------------------------------------------- CSR assembly

class Graph:
    """A CSR adjacency pattern plus a short description of how it was made."""

    def __init__(self, row_ptr: np.ndarray, col_idx: np.ndarray, name: str, info: dict | None = None):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.name = name
        self.info = dict(info or {})

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def __repr__(self) -> str:  # pragma: no cover - cosmetic
        return f"Graph({self.name}, n={self.n}, nnz={self.nnz})"


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Symmetrise, drop self loops and duplicates, and return sorted CSR (row_ptr, col_idx)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.concatenate([u, v])
    b = np.concatenate([v, u])
    key = np.sort(a * np.int64(n) + b)
    if key.shape[0]:
        first = np.empty(key.shape[0], dtype=bool)
        first[0] = True
        np.not_equal(key[1:], key[:-1], out=first[1:])
        key = key[first]
    rows = key // n
    cols = key - rows * n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32)


def largest_component(row_ptr: np.ndarray, col_idx: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Largest connected component, vertices relabelled in ascending original order.

    Returns (row_ptr, col_idx, kept_vertex_ids).  Ties between equally large
    components go to the one holding the smallest vertex id.
    """
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    n = row_ptr.shape[0] - 1
    A = sp.csr_matrix((np.ones(col_idx.shape[0], dtype=np.int8), col_idx, row_ptr), shape=(n, n))
    ncomp, labels = connected_components(A, directed=False)
    if ncomp == 1:
        return row_ptr, col_idx, np.arange(n, dtype=np.int64)
    sizes = np.bincount(labels)
    best = int(np.flatnonzero(sizes == sizes.max())[0])
    keep = np.flatnonzero(labels == best).astype(np.int64)
    newid = np.full(n, -1, dtype=np.int64)
    newid[keep] = np.arange(keep.shape[0], dtype=np.int64)
    deg = np.diff(row_ptr)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    sel = labels[src] == best
    r = newid[src[sel]]
    c = newid[col_idx[sel].astype(np.int64)]
    m = keep.shape[0]
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=rp[1:])
    # rows are already grouped and columns sorted, because relabelling is monotone
    return rp, c.astype(np.int32), keep


# --------------------------------------------------------------------------- structured graphs

def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return Graph(*csr_from_edges(n, i, i + 1), name=f"path{n}")


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return Graph(*csr_from_edges(n, i, (i + 1) % n), name=f"cycle{n}")


def complete(n: int) -> Graph:
    u, v = np.triu_indices(n, 1)
    return Graph(*csr_from_edges(n, u, v), name=f"complete{n}")


def star(n: int) -> Graph:
    """Vertex 0 is the centre, joined to 1..n-1."""
    leaves = np.arange(1, n)
    return Graph(*csr_from_edges(n, np.zeros_like(leaves), leaves), name=f"star{n}")


def hypercube(r: int) -> Graph:
    n = 1 << r
    us, vs = [], []
    x = np.arange(n)
    for b in range(r):
        y = x ^ (1 << b)
        sel = x < y
        us.append(x[sel])
        vs.append(y[sel])
    return Graph(*csr_from_edges(n, np.concatenate(us), np.concatenate(vs)), name=f"hypercube{r}")


def grid2d(nx: int, ny: int) -> Graph:
    """5-point grid; vertex (a, b) with 0<=a<nx, 0<=b<ny has id a*ny + b."""
    idx = np.arange(nx * ny).reshape(nx, ny)
    us = [idx[:-1, :].ravel(), idx[:, :-1].ravel()]
    vs = [idx[1:, :].ravel(), idx[:, 1:].ravel()]
    return Graph(*csr_from_edges(nx * ny, np.concatenate(us), np.concatenate(vs)), name=f"grid{nx}x{ny}")


def grid3d(nx: int, ny: int, nz: int) -> Graph:
    """7-point grid; vertex (a, b, c) has id (a*ny + b)*nz + c."""
    n = nx * ny * nz
    # build CSR directly in sorted order (cheap and memory-light for 128^3)
    idx = np.arange(n, dtype=np.int64).reshape(nx, ny, nz)
    nb = []
    for d, (sa, sb) in enumerate([((slice(1, None), slice(None), slice(None)), (slice(None, -1), slice(None), slice(None))),
                                  ((slice(None), slice(1, None), slice(None)), (slice(None), slice(None, -1), slice(None))),
                                  ((slice(None), slice(None), slice(1, None)), (slice(None), slice(None), slice(None, -1)))]):
        nb.append((idx[sa].ravel(), idx[sb].ravel()))
    u = np.concatenate([a for a, _ in nb])
    v = np.concatenate([b for _, b in nb])
    return Graph(*csr_from_edges(n, u, v), name=f"grid{nx}x{ny}x{nz}")


# --------------------------------------------------------------------------- random graphs

def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, lcc: bool = True, batch: int = 1 << 24) -> Graph:
    """R-MAT graph (Chakrabarti, Zhan, Faloutsos 2004) with 2^scale vertices.

    edge_factor * 2^scale directed samples; sample e picks one quadrant per
    level l with the uniform number uniform01(seed, e*scale + l) (level 0 is the
    most significant bit).  No noise, no vertex permutation.  The result is
    symmetrised, deduplicated, loop-free and (by default) reduced to its largest
    connected component.
    """
    n = 1 << scale
    E = edge_factor * n
    ab, abc = a + b, a + b + c
    us, vs = [], []
    for e0 in range(0, E, batch):
        e = np.arange(e0, min(E, e0 + batch), dtype=np.uint64)
        u = np.zeros(e.shape[0], dtype=np.int64)
        v = np.zeros(e.shape[0], dtype=np.int64)
        for lvl in range(scale):
            x = uniform01(seed, e * np.uint64(scale) + np.uint64(lvl))
            bit = np.int64(1 << (scale - 1 - lvl))
            down = x >= ab                      # quadrants c, d: row bit set
            right = ((x >= a) & (x < ab)) | (x >= abc)   # quadrants b, d: column bit set
            u += down.astype(np.int64) * bit
            v += right.astype(np.int64) * bit
        us.append(u)
        vs.append(v)
    rp, ci = csr_from_edges(n, np.concatenate(us), np.concatenate(vs))
    info = {"scale": scale, "edge_factor": edge_factor, "abcd": (a, b, c, 1 - a - b - c), "seed": seed,
            "n_full": n}
    if lcc:
        rp, ci, keep = largest_component(rp, ci)
        info["lcc"] = True
    return Graph(rp, ci, name=f"rmat{scale}", info=info)


def rgg(n: int, mean_degree: float = 12.0, seed: int = 1, lcc: bool = True) -> Graph:
    """Random geometric graph in the unit square (not a torus).

    Point t has coordinates (uniform01(seed, 2t), uniform01(seed, 2t+1)); two
    points are joined when their distance is at most r = sqrt(mean_degree/(pi n))
    (boundary effects ignored when choosing r).
    """
    from scipy.spatial import cKDTree

    t = np.arange(n, dtype=np.uint64)
    pts = np.stack([uniform01(seed, 2 * t), uniform01(seed, 2 * t + np.uint64(1))], axis=1)
    r = math.sqrt(mean_degree / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    rp, ci = csr_from_edges(n, pairs[:, 0], pairs[:, 1])
    info = {"radius": r, "seed": seed}
    if lcc:
        rp, ci, _ = largest_component(rp, ci)
    g = Graph(rp, ci, name=f"rgg{n}", info=info)
    g.info["mean_degree"] = g.nnz / max(g.n, 1)
    return g


def erdos_renyi(n: int, mean_degree: float = 8.0, seed: int = 1, lcc: bool = True) -> Graph:
    """G(n, M) stand-in for G(n, p = mean_degree/(n-1)): M = round(n*mean_degree/2) uniform pairs."""
    M = int(round(n * mean_degree / 2))
    e = np.arange(M, dtype=np.uint64)
    u = np.minimum((uniform01(seed, 2 * e) * n).astype(np.int64), n - 1)
    v = np.minimum((uniform01(seed, 2 * e + np.uint64(1)) * n).astype(np.int64), n - 1)
    rp, ci = csr_from_edges(n, u, v)
    if lcc:
        rp, ci, _ = largest_component(rp, ci)
    return Graph(rp, ci, name=f"er{n}")


def watts_strogatz(n: int, k: int = 10, p: float = 0.1, seed: int = 1, lcc: bool = True) -> Graph:
    """Ring lattice with k/2 neighbours per side; each lattice edge (t, t+j) is
    rewired to (t, w) with probability p, w uniform (loops/duplicates dropped)."""
    half = k // 2
    t = np.repeat(np.arange(n, dtype=np.int64), half)
    j = np.tile(np.arange(1, half + 1, dtype=np.int64), n)
    v = (t + j) % n
    ctr = np.arange(t.shape[0], dtype=np.uint64)
    rew = uniform01(seed, 2 * ctr) < p
    w = np.minimum((uniform01(seed, 2 * ctr + np.uint64(1)) * n).astype(np.int64), n - 1)
    v = np.where(rew, w, v)
    rp, ci = csr_from_edges(n, t, v)
    if lcc:
        rp, ci, _ = largest_component(rp, ci)
    return Graph(rp, ci, name=f"ws{n}")


def grid2d_near(n: int) -> Graph:
    """2D grid with ceil(sqrt(n)) x floor(n / ceil(sqrt(n))) vertices."""
    a = int(math.ceil(math.sqrt(n)))
    b = max(1, n // a)
    return grid2d(a, b)


def batch_family(G: int = 256, nmin: int = 1000, nmax: int = 200000, seed: int = 1) -> list[Graph]:
    """Heterogeneous batch: graph g has n_g = round(exp(U(ln nmin, ln nmax))) drawn from
    stream (seed, g); family g mod 3 is ER (mean degree 8) / 2D grid / WS(k=10, p=0.1)."""
    out = []
    for g in range(G):
        s = stream_seed(seed, g)
        u = float(uniform01(s, 0))
        ng = int(round(math.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))))
        fam = g % 3
        if fam == 0:
            out.append(erdos_renyi(ng, 8.0, seed=s))
        elif fam == 1:
            out.append(grid2d_near(ng))
        else:
            out.append(watts_strogatz(ng, 10, 0.1, seed=s))
    return out


# --------------------------------------------------------------------------- edge weights

def edge_weights(g: Graph, seed: int = 1, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Positive weights aligned with g.col_idx for the weighted Laplacian: edge {u, v} gets
    lo + (hi - lo) * uniform01(seed, min(u, v) * n + max(u, v)), so both stored directions of an
    edge carry the same weight."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    cols = g.col_idx.astype(np.int64)
    key = np.minimum(rows, cols) * np.int64(g.n) + np.maximum(rows, cols)
    return lo + (hi - lo) * uniform01(seed, key.astype(np.uint64))


# --------------------------------------------------------------------------- start vector

def start_vector(n: int, seed: int = 1) -> np.ndarray:
    """The column u_1 of U_{k0} (k0 = 1): x_t = 2*uniform01(seed, t) - 1, centred so that it is
    orthogonal to the all-ones vector, and scaled to unit 2-norm (the REQUIRE clause of
    Algorithm 2 asks for an orthonormal start basis orthogonal to 1)."""
    x = 2.0 * uniform01(seed, np.arange(n, dtype=np.uint64)) - 1.0
    x -= x.mean()
    x -= x.mean()
    return x / np.linalg.norm(x)


# --------------------------------------------------------------------------- named workloads

def workload(name: str) -> Graph:
    """The named synthetic workloads used by tests and the benchmark."""
    if name == "grid100x100":
        return grid2d(100, 100)
    if name.startswith("rmat"):
        return rmat(int(name[4:]))
    if name == "grid128^3":
        return grid3d(128, 128, 128)
    if name == "rgg4M":
        return rgg(4_000_000, 12.0, seed=1)
    raise KeyError(name)


# --------------------------------------------------------------------------- GPU generation (large graphs)

def _splitmix64_torch(seed: int, counter):
    """splitmix64(seed, counter) on int64 torch tensors: wrapping multiply, logical right shifts."""
    import torch

    def u64(v):  # reinterpret an unsigned 64-bit constant as int64
        return v - (1 << 64) if v >= (1 << 63) else v

    def lsr(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    z = torch.full_like(counter, u64(seed & 0xFFFFFFFFFFFFFFFF)) + (counter + 1) * u64(0x9E3779B97F4A7C15)
    z = (z ^ lsr(z, 30)) * u64(0xBF58476D1CE4E5B9)
    z = (z ^ lsr(z, 27)) * u64(0x94D049BB133111EB)
    return z ^ lsr(z, 31)


def _uniform01_torch(seed: int, counter):
    return _splitmix64_torch(seed, counter).__rshift__(11).bitwise_and((1 << 53) - 1).double() * (1.0 / 9007199254740992.0)


def rmat_gpu(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
             seed: int = 1, device: str = "cuda", batch: int = 1 << 25):
    """The graph of rmat(scale, ...) (same draws, same symmetrisation, deduplication, largest
    component and relabelling) built with torch on the GPU.  Returns (row_ptr, col_idx) as
    device tensors (int64, int32)."""
    import torch
    n = 1 << scale
    E = edge_factor * n
    ab, abc = a + b, a + b + c
    keys = []
    for e0 in range(0, E, batch):
        e = torch.arange(e0, min(E, e0 + batch), dtype=torch.int64, device=device)
        u = torch.zeros_like(e)
        v = torch.zeros_like(e)
        for lvl in range(scale):
            x = _uniform01_torch(seed, e * scale + lvl)
            bit = 1 << (scale - 1 - lvl)
            down = x >= ab
            right = ((x >= a) & (x < ab)) | (x >= abc)
            u += down.to(torch.int64) * bit
            v += right.to(torch.int64) * bit
        keep = u != v
        u, v = u[keep], v[keep]
        keys.append(u * n + v)
        keys.append(v * n + u)
        del e, x, down, right
    return _csr_lcc_gpu(torch.cat(keys), n)


def _csr_lcc_gpu(keys, n):
    """CSR (row_ptr int64, col_idx int32, device tensors) of the largest connected component of the
    graph whose directed edge keys u * n + v (both directions present) are given, with the same
    deduplication, tie rule and ascending relabelling as largest_component()."""
    import torch
    device = keys.device
    key = torch.unique(keys)                     # sorted, deduplicated
    del keys
    rows = key // n
    cols = key - rows * n
    del key
    # connected components by min-label propagation (labels converge to the component minimum)
    lab = torch.arange(n, dtype=torch.int64, device=device)
    while True:
        nl = lab.clone()
        nl.scatter_reduce_(0, rows, lab[cols], reduce="amin")
        nl = torch.minimum(nl, nl[nl])           # pointer jumping
        if torch.equal(nl, lab):
            break
        lab = nl
    present = torch.zeros(n, dtype=torch.bool, device=device)
    present[rows] = True
    counts = torch.bincount(lab[present], minlength=n)
    best = int(torch.argmax(counts).item())      # largest component; ties -> smallest label (= smallest id)
    keepv = lab == best
    keepv &= present if counts[best] > 1 else keepv
    newid = torch.full((n,), -1, dtype=torch.int64, device=device)
    kept = torch.nonzero(keepv).flatten()
    newid[kept] = torch.arange(kept.numel(), dtype=torch.int64, device=device)
    sel = keepv[rows]
    r2 = newid[rows[sel]]
    c2 = newid[cols[sel]]
    m = kept.numel()
    rp = torch.zeros(m + 1, dtype=torch.int64, device=device)
    rp[1:] = torch.cumsum(torch.bincount(r2, minlength=m), 0)
    return rp, c2.to(torch.int32)


def rgg_gpu(n: int, mean_degree: float = 12.0, seed: int = 1, device: str = "cuda", batch: int = 1 << 22):
    """The graph of rgg(n, mean_degree, seed) (same points, pairs at distance <= r, largest
    component, ascending relabelling) built with torch on the GPU from a cell list: the unit
    square is cut into square cells of side >= r, so every pair within distance r lies in the
    same or in adjacent cells.  Returns (row_ptr, col_idx) as device tensors (int64, int32)."""
    import torch
    r = math.sqrt(mean_degree / (math.pi * n))
    t = torch.arange(n, dtype=torch.int64, device=device)
    px = _uniform01_torch(seed, 2 * t)
    py = _uniform01_torch(seed, 2 * t + 1)
    nc = max(1, int(math.floor(1.0 / r)))        # cells per side, side 1/nc >= r
    cx = torch.clamp((px * nc).to(torch.int64), max=nc - 1)
    cy = torch.clamp((py * nc).to(torch.int64), max=nc - 1)
    cell = cx * nc + cy
    order = torch.argsort(cell)
    cell_sorted = cell[order]
    start = torch.zeros(nc * nc + 1, dtype=torch.int64, device=device)
    start[1:] = torch.cumsum(torch.bincount(cell_sorted, minlength=nc * nc), 0)
    r2 = r * r
    keys = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for b0 in range(0, n, batch):
                i = order[b0:b0 + batch]                  # points, in cell order
                ncx, ncy = cx[i] + dx, cy[i] + dy
                ok = (ncx >= 0) & (ncx < nc) & (ncy >= 0) & (ncy < nc)
                i = i[ok]
                c2 = (ncx * nc + ncy)[ok]
                cnt = start[c2 + 1] - start[c2]
                ii = torch.repeat_interleave(i, cnt)
                off = torch.repeat_interleave(start[c2] - torch.cumsum(cnt, 0) + cnt, cnt)
                jj = order[off + torch.arange(ii.numel(), dtype=torch.int64, device=device)]
                d2 = (px[ii] - px[jj]) ** 2 + (py[ii] - py[jj]) ** 2
                keep = (d2 <= r2) & (ii < jj)
                u, v = ii[keep], jj[keep]
                keys.append(u * n + v)
                keys.append(v * n + u)
                del ii, jj, off, d2, keep
    return _csr_lcc_gpu(torch.cat(keys), n)
