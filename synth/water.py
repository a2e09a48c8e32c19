"""Water-like block-sparse symmetric matrices, seeded and synthetic.

The paper measured the submatrix method on Kohn-Sham matrices of bulk water
(Section 3, Fig. 2 and the record run that follows it); neither those systems
nor their basis sets are available, so these generators stand in for them with
the shapes and value distributions the workloads call for:

* one "molecule" = one block row/column of size ``b`` (6 or 23 orbitals);
* molecules sit on a jittered simple-cubic lattice in a periodic box (or in a
  water/vacuum slab), with minimum-image centre distances ``d_ij``;
* diagonal block ``i`` is ``Q diag(eps) Q^T`` with a Haar-random orthogonal
  ``Q``; the first ``b // 2`` on-site energies are drawn from N(-0.5, 0.05)
  (occupied band) and the rest from N(+0.5, 0.05) (virtual band), giving a gap
  around mu = 0;
* for ``i < j`` with ``d_ij < r_c`` the block ``H_ij`` has i.i.d. entries
  N(0, 0.1) * exp(-d_ij / ell) and ``H_ji = H_ij^T``.

The off-diagonal entries come from a counter-based generator keyed by
(seed, i, j, entry) so that a pair's block is the same in every snapshot of a
trajectory and does not depend on which other pairs exist.

Output format (shared by the oracle and the library): block-CSC with the full
symmetric pattern, ``col_ptr`` (int64, length B+1), ``row_idx`` (int32, sorted
within each column), and ``values`` (float64) holding the blocks in CSC order,
each block ``b_r x b_c`` stored column-major.

Nothing here filters, shifts, or computes any matrix function.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Iterator

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


@dataclasses.dataclass
class BlockCSC:
    """A block-sparse symmetric matrix in block-CSC form (see module docstring)."""

    block_size: np.ndarray  # int32 [B]
    col_ptr: np.ndarray  # int64 [B+1]
    row_idx: np.ndarray  # int32 [nnzb]
    values: np.ndarray  # float64, blocks concatenated, column-major each
    positions: np.ndarray | None = None  # float64 [B, 3], Angstrom
    box: np.ndarray | None = None  # float64 [3], Angstrom
    n_occ: int = 0  # number of occupied orbitals (b // 2 per molecule)
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_blocks(self) -> int:
        return int(self.block_size.shape[0])

    @property
    def n(self) -> int:
        return int(self.block_size.sum())

    @property
    def nnzb(self) -> int:
        return int(self.row_idx.shape[0])


# --------------------------------------------------------------------------
# counter-based normals (SplitMix64 finaliser + Box-Muller)
# --------------------------------------------------------------------------

def _splitmix64(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def keyed_normals(seed: int, i: np.ndarray, j: np.ndarray, count: int) -> np.ndarray:
    """Standard normals N(0,1) of shape [len(i), count], a pure function of (seed, i, j, k)."""
    i = np.asarray(i, dtype=np.uint64).reshape(-1, 1)
    j = np.asarray(j, dtype=np.uint64).reshape(-1, 1)
    k = np.arange(count, dtype=np.uint64).reshape(1, -1)
    with np.errstate(over="ignore"):
        key = _splitmix64(np.uint64(seed & 0xFFFFFFFF) * np.uint64(0x100000001B3) ^ _splitmix64((i << np.uint64(32)) | j))
        h1 = _splitmix64(key + np.uint64(2) * k)
        h2 = _splitmix64(key + np.uint64(2) * k + np.uint64(1))
    u1 = (h1 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def _haar_orthogonal(rng: np.random.Generator, b: int) -> np.ndarray:
    g = rng.standard_normal((b, b))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def spectrum_matrix(n: int, eigs, seed: int) -> np.ndarray:
    """Dense symmetric ``Q diag(eigs) Q^T`` with a seeded Haar-random ``Q`` (test input)."""
    rng = np.random.default_rng(seed)
    q = _haar_orthogonal(rng, n)
    a = (q * np.asarray(eigs, dtype=np.float64)[None, :]) @ q.T
    return 0.5 * (a + a.T)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def lattice_positions(n_mol: int, spacing: float, jitter: float, rng: np.random.Generator):
    """Jittered simple-cubic placement: box L = spacing * n_mol^(1/3), ceil(n_mol^(1/3)) sites per side."""
    box_len = spacing * n_mol ** (1.0 / 3.0)
    per_side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    grid = box_len / per_side
    sites = np.stack(np.meshgrid(*(np.arange(per_side),) * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    pick = rng.permutation(sites.shape[0])[:n_mol]
    pos = (sites[pick] + 0.5) * grid
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape)
    return pos, np.array([box_len] * 3)


def slab_positions(n_mol: int, box, rho0: float, width: float, hard_core: float, rng: np.random.Generator):
    """Water/vacuum slab: z density rho0 * 0.5*[tanh((z-z1)/w) - tanh((z-z2)/w)], hard-core rejection."""
    box = np.asarray(box, dtype=np.float64)
    thickness = n_mol / (rho0 * box[0] * box[1])
    z1 = 0.5 * box[2] - 0.5 * thickness
    z2 = 0.5 * box[2] + 0.5 * thickness
    pos = np.empty((n_mol, 3))
    count = 0
    hc2 = hard_core * hard_core
    while count < n_mol:
        cand = rng.uniform(0.0, 1.0, size=(4096, 4))
        cand_pos = cand[:, :3] * box
        prof = 0.5 * (np.tanh((cand_pos[:, 2] - z1) / width) - np.tanh((cand_pos[:, 2] - z2) / width))
        cand_pos = cand_pos[cand[:, 3] < prof]
        for p in cand_pos:
            if count:
                dv = pos[:count] - p
                dv -= box * np.round(dv / box)
                if np.min(np.einsum("ij,ij->i", dv, dv)) < hc2:
                    continue
            pos[count] = p
            count += 1
            if count == n_mol:
                break
    return pos, box


def _pairs_within(pos: np.ndarray, box: np.ndarray, r_c: float):
    """All pairs i < j with minimum-image centre distance < r_c (chunked brute force)."""
    n = pos.shape[0]
    out_i, out_j, out_d = [], [], []
    chunk = max(1, 4_000_000 // max(n, 1))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        dv = pos[s:e, None, :] - pos[None, :, :]
        dv -= box * np.round(dv / box)
        d = np.sqrt(np.einsum("abk,abk->ab", dv, dv))
        ii, jj = np.nonzero(d < r_c)
        gi = ii + s
        keep = gi < jj
        out_i.append(gi[keep])
        out_j.append(jj[keep])
        out_d.append(d[ii[keep], jj[keep]])
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_d)


# --------------------------------------------------------------------------
# assembly
# --------------------------------------------------------------------------

def _diag_blocks(n_mol: int, b: int, rng: np.random.Generator, occ=(-0.5, 0.05), virt=(0.5, 0.05)):
    n_occ = b // 2
    blocks = np.empty((n_mol, b, b))
    for m in range(n_mol):
        q = _haar_orthogonal(rng, b)
        eps = np.concatenate([rng.normal(occ[0], occ[1], n_occ), rng.normal(virt[0], virt[1], b - n_occ)])
        a = (q * eps[None, :]) @ q.T
        blocks[m] = 0.5 * (a + a.T)
    return blocks


def _assemble(pos, box, b, diag, seed, r_c, ell, sigma, pairs=None) -> BlockCSC:
    n_mol = pos.shape[0]
    if pairs is not None:  # a fixed pattern: the given pairs at their current distances
        pi, pj = pairs
        dv = pos[pi] - pos[pj]
        dv -= box * np.round(dv / box)
        d = np.sqrt(np.einsum("ak,ak->a", dv, dv))
    elif np.isfinite(r_c):
        pi, pj, d = _pairs_within(pos, box, r_c)
    else:
        pi, pj = np.triu_indices(n_mol, k=1)
        dv = pos[pi] - pos[pj]
        dv -= box * np.round(dv / box)
        d = np.sqrt(np.einsum("ak,ak->a", dv, dv))
    amp = sigma * np.exp(-d / ell)
    m = keyed_normals(seed, pi, pj, b * b).reshape(-1, b, b) * amp[:, None, None]
    rows = np.concatenate([np.arange(n_mol), pi, pj]).astype(np.int64)
    cols = np.concatenate([np.arange(n_mol), pj, pi]).astype(np.int64)
    blocks = np.concatenate([diag, m, m.transpose(0, 2, 1)], axis=0)
    order = np.lexsort((rows, cols))
    rows, cols, blocks = rows[order], cols[order], blocks[order]
    col_ptr = np.zeros(n_mol + 1, dtype=np.int64)
    col_ptr[1:] = np.cumsum(np.bincount(cols, minlength=n_mol))
    values = np.ascontiguousarray(blocks.transpose(0, 2, 1)).reshape(-1)  # column-major per block
    return BlockCSC(
        block_size=np.full(n_mol, b, dtype=np.int32),
        col_ptr=col_ptr,
        row_idx=rows.astype(np.int32),
        values=values,
        positions=pos,
        box=np.asarray(box, dtype=np.float64),
        n_occ=n_mol * (b // 2),
    )


def make_lattice_system(n_mol: int, b: int, r_c: float, ell: float, seed: int,
                        spacing: float = 3.1, jitter: float = 0.3, sigma: float = 0.1) -> BlockCSC:
    """Bulk-water-like system on a jittered periodic cubic lattice."""
    rng = np.random.default_rng(seed)
    pos, box = lattice_positions(n_mol, spacing, jitter, rng)
    diag = _diag_blocks(n_mol, b, rng)
    sysm = _assemble(pos, box, b, diag, seed, r_c, ell, sigma)
    sysm.meta = dict(kind="lattice", n_mol=n_mol, b=b, r_c=r_c, ell=ell, seed=seed)
    return sysm


def make_overlap_system(n_mol: int, b: int, r_c: float, ell: float, seed: int, spacing: float = 3.1,
                        jitter: float = 0.3, sigma: float = 0.05, diag_spread: float = 0.05) -> BlockCSC:
    """Overlap-like symmetric positive definite matrix with the lattice system's block pattern:
    diagonal blocks I + diag_spread * (G + G^T)/2 (G standard normal), off-diagonal blocks
    N(0, sigma) exp(-d/ell) as in the Hamiltonian stand-in.  With the defaults every Gershgorin
    disc of the water-like patterns stays well right of zero (checked where it is used)."""
    rng = np.random.default_rng(seed)
    pos, box = lattice_positions(n_mol, spacing, jitter, rng)
    g = rng.standard_normal((n_mol, b, b))
    diag = np.eye(b)[None, :, :] + diag_spread * 0.5 * (g + g.transpose(0, 2, 1))
    sysm = _assemble(pos, box, b, diag, seed, r_c, ell, sigma)
    sysm.meta = dict(kind="overlap", n_mol=n_mol, b=b, r_c=r_c, ell=ell, seed=seed)
    return sysm


def make_nonorth_pair(n_mol: int, b: int, r_c: float, ell: float, seed: int, spacing: float = 3.1,
                      jitter: float = 0.3, sigma_h: float = 0.1, sigma_s: float = 0.05,
                      diag_spread: float = 0.05):
    """A Kohn-Sham-like H and an overlap-like S of one molecular geometry, in a non-orthogonal
    basis: both on the block pattern of the pairs within r_c.  H as in the lattice system
    (two bands of on-site energies, off-diagonal N(0, sigma_h) exp(-d/ell)); S with diagonal
    blocks I + diag_spread (G + G^T)/2 and off-diagonal N(0, sigma_s) exp(-d/ell) from a
    second key stream, so that S is not a multiple of H off the diagonal.  Returns (H, S)
    as two BlockCSC with identical patterns."""
    rng = np.random.default_rng(seed)
    pos, box = lattice_positions(n_mol, spacing, jitter, rng)
    diag_h = _diag_blocks(n_mol, b, rng)
    g = rng.standard_normal((n_mol, b, b))
    diag_s = np.eye(b)[None, :, :] + diag_spread * 0.5 * (g + g.transpose(0, 2, 1))
    pairs = _pairs_within(pos, box, r_c)[:2] if np.isfinite(r_c) else np.triu_indices(n_mol, k=1)
    h = _assemble(pos, box, b, diag_h, seed, r_c, ell, sigma_h, pairs=pairs)
    s = _assemble(pos, box, b, diag_s, seed + 0x5A17, r_c, ell, sigma_s, pairs=pairs)
    h.meta = dict(kind="nonorth_h", n_mol=n_mol, b=b, r_c=r_c, ell=ell, seed=seed)
    s.meta = dict(kind="nonorth_s", n_mol=n_mol, b=b, r_c=r_c, ell=ell, seed=seed)
    return h, s


def make_slab_system(n_mol: int, b: int, r_c: float, ell: float, seed: int, box=(50.0, 50.0, 200.0),
                     width: float = 8.0, hard_core: float = 2.0, sigma: float = 0.1) -> BlockCSC:
    """Water/vacuum slab: bulk density 1/3.1^3 per cubic Angstrom ramping to zero across two interfaces."""
    rng = np.random.default_rng(seed)
    pos, boxv = slab_positions(n_mol, box, 1.0 / 3.1 ** 3, width, hard_core, rng)
    diag = _diag_blocks(n_mol, b, rng)
    sysm = _assemble(pos, boxv, b, diag, seed, r_c, ell, sigma)
    sysm.meta = dict(kind="slab", n_mol=n_mol, b=b, r_c=r_c, ell=ell, seed=seed)
    return sysm


def md_trajectory(n_mol: int, b: int, r_c: float, ell: float, seed: int, n_snap: int,
                  step_sigma: float = 0.05, fixed_pattern: bool = False) -> Iterator[BlockCSC]:
    """Snapshots of a lattice system whose positions take cumulative N(0, step_sigma) steps.

    Diagonal blocks stay fixed; each pair's off-diagonal block keeps its random
    pattern and only its amplitude follows the distance, so matrices evolve
    smoothly.  The block pattern is recomputed per snapshot, or, with
    ``fixed_pattern``, is the pairs within r_c at the first snapshot for the
    whole trajectory (one library context can then take every snapshot).
    """
    rng = np.random.default_rng(seed)
    pos, box = lattice_positions(n_mol, 3.1, 0.3, rng)
    diag = _diag_blocks(n_mol, b, rng)
    step_rng = np.random.default_rng(seed + 7919)
    pairs = _pairs_within(pos, box, r_c)[:2] if fixed_pattern else None
    for s in range(n_snap):
        if s:
            pos = pos + step_rng.normal(0.0, step_sigma, size=pos.shape)
            pos = np.mod(pos, box)
        sysm = _assemble(pos, box, b, diag, seed, r_c, ell, 0.1, pairs=pairs)
        sysm.meta = dict(kind="md", n_mol=n_mol, b=b, r_c=r_c, ell=ell, seed=seed, snapshot=s)
        yield sysm


def make_mixed_block_system(block_sizes, r_c: float, ell: float, seed: int, spacing: float = 3.1,
                            jitter: float = 0.3, sigma: float = 0.1) -> BlockCSC:
    """Lattice system whose molecules have different block sizes (small systems only).

    Molecule i has ``block_sizes[i]`` orbitals; its on-site energies split into
    the two bands as for uniform blocks; off-diagonal blocks are
    ``b_i x b_j`` with the same keyed entries and decay.
    """
    sizes = np.asarray(block_sizes, dtype=np.int64)
    n_mol = sizes.shape[0]
    rng = np.random.default_rng(seed)
    pos, box = lattice_positions(n_mol, spacing, jitter, rng)
    diag = []
    for b in sizes:
        diag.append(_diag_blocks(1, int(b), rng)[0])
    if np.isfinite(r_c):
        pi, pj, d = _pairs_within(pos, box, r_c)
    else:
        pi, pj = np.triu_indices(n_mol, k=1)
        dv = pos[pi] - pos[pj]
        dv -= box * np.round(dv / box)
        d = np.sqrt(np.einsum("ak,ak->a", dv, dv))
    bmax = int(sizes.max())
    g = keyed_normals(seed, pi, pj, bmax * bmax).reshape(-1, bmax, bmax)
    entries = {(i, i): diag[i] for i in range(n_mol)}
    for t in range(pi.shape[0]):
        i, j = int(pi[t]), int(pj[t])
        m = g[t, : sizes[i], : sizes[j]] * sigma * np.exp(-d[t] / ell)
        entries[(i, j)] = m
        entries[(j, i)] = m.T
    col_ptr = np.zeros(n_mol + 1, dtype=np.int64)
    rows, vals = [], []
    for j in range(n_mol):
        rj = sorted(i for (i, jj) in entries if jj == j)
        for i in rj:
            rows.append(i)
            vals.append(entries[(i, j)].T.reshape(-1))
        col_ptr[j + 1] = len(rows)
    sysm = BlockCSC(block_size=sizes.astype(np.int32), col_ptr=col_ptr, row_idx=np.asarray(rows, dtype=np.int32),
                    values=np.concatenate(vals), positions=pos, box=box, n_occ=int(np.sum(sizes // 2)))
    sysm.meta = dict(kind="mixed", n_mol=n_mol, r_c=r_c, ell=ell, seed=seed)
    return sysm


# Named workloads. Each entry gives the generator arguments and the method
# settings (filter threshold eps, fixed mu or electron count).
WORKLOADS = {
    # 32 molecules, 6x6 blocks, N = 192: fixed mu = 0, no filtering
    "water32": dict(gen="lattice", n_mol=32, b=6, r_c=5.0, ell=1.5, seed=1001, eps=0.0, mu=0.0),
    # same, complete pattern: one submatrix equals the whole matrix
    "water32_full": dict(gen="lattice", n_mol=32, b=6, r_c=math.inf, ell=1.5, seed=1001, eps=0.0, mu=0.0),
    # 1024 molecules, 6x6 blocks, N = 6144: bisection to trace(D) = 3072
    "water1024": dict(gen="lattice", n_mol=1024, b=6, r_c=6.0, ell=1.5, seed=1002, eps=1e-5, n_e=3072.0),
    # 4096 molecules, 23x23 blocks, N = 94208: fixed mu = 0
    "water4096x23": dict(gen="lattice", n_mol=4096, b=23, r_c=7.0, ell=2.0, seed=1003, eps=1e-6, mu=0.0),
    # 6000-molecule water/vacuum slab, 6x6 blocks, wide cutoff: 20-step bisection to 3 * 6000
    "slab6000": dict(gen="slab", n_mol=6000, b=6, r_c=15.3, ell=3.0, seed=1004, eps=1e-5, n_e=18000.0, max_steps=20),
    # MD-like trajectory of the 1024-molecule system (200 snapshots)
    "md1024": dict(gen="md", n_mol=1024, b=6, r_c=6.0, ell=1.5, seed=1005, eps=1e-5, n_e=3072.0, n_snap=200),
}


def make_workload(name: str, **override) -> BlockCSC:
    """Build a named workload (not the trajectory one); ``override`` replaces generator arguments."""
    w = dict(WORKLOADS[name])
    w.update(override)
    if w["gen"] == "lattice":
        s = make_lattice_system(w["n_mol"], w["b"], w["r_c"], w["ell"], w["seed"])
    elif w["gen"] == "slab":
        s = make_slab_system(w["n_mol"], w["b"], w["r_c"], w["ell"], w["seed"])
    else:
        raise ValueError(f"workload {name} is a trajectory; use md_trajectory")
    s.meta.update(name=name, eps=w.get("eps", 0.0), mu=w.get("mu"), n_e=w.get("n_e"))
    return s
