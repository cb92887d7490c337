"""Seeded synthetic inputs for OMM solves: atomic-orbital-like H, S, W0 and block patterns.

This module only *generates inputs*.  It holds none of the method's arithmetic
(no shift, no functional, no gradient, no line search, no filtering): both the
FP64 oracle and the CUDA library consume the arrays it returns.

Recipe (the paper's BN/DZP SIESTA matrices are not available; these stand in
for them with the same structure: equal atom blocks, short-ranged H and S,
an insulating gap, n/m = 1/4 occupied orbitals, localised W patterns):

* Atoms on a cubic grid of spacing 2.5 A, index I = (ix*ny + iy)*nz + iz,
  each coordinate jittered by U(-0.2, 0.2) A.  Open boundaries.
* 8 orbitals per atom (block size b_BF = 8); 2 occupied orbitals per atom
  (b_WF = b_BF * n/m = 2, the paper's default block-size rule, Table 1).
* Onsite H block: diagonal (-5,-5,+5,+5,+5,+5,+5,+5) eV + N(0, 0.3) per orbital.
* For every atom pair I<J with r_IJ <= 5 A (inclusive), in lexicographic (I, J)
  order: H_IJ = 0.8 exp(-r/1.5) R_IJ with R_IJ ~ N(0,1)^{8x8};
  S_IJ = 0.15 exp(-r/1.2) B_IJ with B_IJ ~ U(-1,1)^{8x8}/8;  H_JI = H_IJ^T,
  S_JI = S_IJ^T; S_II = I_8.  Row sums of |S_IJ| stay well below 1, so S is
  strictly diagonally dominant and hence SPD.
* Draw order from one PCG64 stream seeded with `seed`: jitter (N x 3), onsite
  noise (N x 8), all R blocks (npairs x 8 x 8), all B blocks (npairs x 8 x 8).
* W0 from a second PCG64 stream seeded with seed + 10**6, drawn as an (n, m)
  C-ordered array (orbital-major, i.e. W in column-major order):
  dense W0 ~ N(0, 1/sqrt(m)); localised W0 keeps only entries whose basis
  atom lies within R_C of the orbital's host atom (orbital j lives on atom
  j // 2) and rescales column j by sqrt(m / nnz_j), i.e. sigma_j = 1/sqrt(nnz_j).
* Kinetic-energy matrix T (for the preconditioner of Eq. 6), on the pairs of
  H and S: onsite diagonal (2, 2, 0.5, 20, 50, 100, 200, 400) eV + N(0, 0.05)
  per orbital -- small on the two occupied-like orbitals and on one low
  unoccupied orbital (the gap stays), a wide range on the others, as for the
  polarisation orbitals of a DZP basis -- and off-site
  T_IJ = 0.05 exp(-r/1.2) K_IJ with K_IJ ~ U(-1,1)^{8x8}/8, T_JI = T_IJ^T.
  Off-site row sums of |T| stay below 0.05 eV < 0.5 eV - 4 sigma, so T is SPD.
  Drawn from a third PCG64 stream seeded with seed + 2*10**6: onsite noise
  (N x 8), then all K blocks (npairs x 8 x 8) in pair order; H, S and W0 are
  unchanged by it.  The kinetic workload's Hamiltonian is H + T (spectrum
  widened to ~400 eV above a gap of a few eV).
* MD trajectories (the pattern update and extrapolation of W between MD
  steps): make_md_system places the atoms at grid + jitter + t * step * v,
  with the jitter and onsite noise drawn as in make_system and one velocity
  v ~ N(0,1)^3 per atom from a PCG64 stream seeded with seed + 3*10**6.  Its
  pair blocks are keyed by the pair: R_IJ, then B_IJ, from a PCG64 stream
  seeded with (seed, I, J), so H and S change smoothly with the positions and
  a pair entering the 5 A cutoff brings its own block (small at the cutoff).
* Batched systems: N atoms = round(exp(U(ln 32, ln 384))) drawn from a PCG64
  stream seeded with the batch seed; the first N sites of the ceil(N^(1/3))^3
  grid in index order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ORB_PER_ATOM = 8
OCC_PER_ATOM = 2
GRID_SPACING = 2.5
JITTER = 0.2
HS_CUTOFF = 5.0
W_RADIUS = 6.0
ONSITE = np.array([-5.0, -5.0, 5.0, 5.0, 5.0, 5.0, 5.0, 5.0])
ONSITE_SIGMA = 0.3
W0_SEED_OFFSET = 10 ** 6
T_SEED_OFFSET = 2 * 10 ** 6
KINETIC_ONSITE = np.array([2.0, 2.0, 0.5, 20.0, 50.0, 100.0, 200.0, 400.0])
KINETIC_SIGMA = 0.05


@dataclass
class System:
    """One synthetic system.  Blocks are 8x8, row-major inside each block."""

    seed: int
    positions: np.ndarray          # (N, 3) Angstrom
    onsite_H: np.ndarray           # (N, 8, 8)
    pairs: np.ndarray              # (npairs, 2) int64, I < J, lexicographic
    pair_r: np.ndarray             # (npairs,)
    H_pair: np.ndarray             # (npairs, 8, 8) block (I, J)
    S_pair: np.ndarray             # (npairs, 8, 8) block (I, J)
    _bsr_cache: dict = field(default_factory=dict, repr=False)

    @property
    def natoms(self) -> int:
        return self.positions.shape[0]

    @property
    def m(self) -> int:
        return self.natoms * ORB_PER_ATOM

    @property
    def n(self) -> int:
        return self.natoms * OCC_PER_ATOM

    # ---------------------------------------------------------------- dense
    def dense_H(self) -> np.ndarray:
        return _assemble_dense(self.natoms, self.onsite_H, self.pairs, self.H_pair)

    def dense_S(self) -> np.ndarray:
        eye = np.broadcast_to(np.eye(ORB_PER_ATOM), (self.natoms, ORB_PER_ATOM, ORB_PER_ATOM))
        return _assemble_dense(self.natoms, eye, self.pairs, self.S_pair)

    def dense_T(self) -> np.ndarray:
        """Kinetic-energy matrix on the pattern of H and S (eV), symmetric positive definite."""
        rng = np.random.Generator(np.random.PCG64(self.seed + T_SEED_OFFSET))
        N = self.natoms
        diag = KINETIC_ONSITE[None, :] + rng.normal(0.0, KINETIC_SIGMA, size=(N, ORB_PER_ATOM))
        onsite = np.zeros((N, ORB_PER_ATOM, ORB_PER_ATOM))
        idx = np.arange(ORB_PER_ATOM)
        onsite[:, idx, idx] = diag
        K = rng.uniform(-1.0, 1.0, size=(self.pairs.shape[0], ORB_PER_ATOM, ORB_PER_ATOM)) / ORB_PER_ATOM
        T_pair = (0.05 * np.exp(-self.pair_r / 1.2))[:, None, None] * K
        return _assemble_dense(N, onsite, self.pairs, T_pair)

    def dense_H_kinetic(self) -> np.ndarray:
        """Hamiltonian of the kinetic workload: H + T (a wide, kinetic-dominated spectrum)."""
        return self.dense_H() + self.dense_T()

    # ---------------------------------------------------------------- block CSR
    def bsr(self):
        """Block-CSR of H and S on the geometric pattern (r_IJ <= 5 A).

        Returns (rowptr int64[N+1], col int32[nnzb], H_vals (nnzb,8,8),
        S_vals (nnzb,8,8)); columns sorted within each block row, diagonal
        block included.
        """
        if "hs" in self._bsr_cache:
            return self._bsr_cache["hs"]
        N = self.natoms
        I = np.concatenate([np.arange(N), self.pairs[:, 0], self.pairs[:, 1]])
        J = np.concatenate([np.arange(N), self.pairs[:, 1], self.pairs[:, 0]])
        Hb = np.concatenate([self.onsite_H, self.H_pair, self.H_pair.transpose(0, 2, 1)])
        eye = np.broadcast_to(np.eye(ORB_PER_ATOM), (N, ORB_PER_ATOM, ORB_PER_ATOM))
        Sb = np.concatenate([eye, self.S_pair, self.S_pair.transpose(0, 2, 1)])
        order = np.lexsort((J, I))
        I, J = I[order], J[order]
        rowptr = np.zeros(N + 1, dtype=np.int64)
        np.add.at(rowptr, I + 1, 1)
        rowptr = np.cumsum(rowptr)
        out = (rowptr, J.astype(np.int32), np.ascontiguousarray(Hb[order]),
               np.ascontiguousarray(Sb[order]))
        self._bsr_cache["hs"] = out
        return out

    def w_pattern(self, radius: float = W_RADIUS):
        """Localisation pattern of W in 8x2 blocks (basis atom I, host atom J).

        Block (I, J) is allowed iff r_IJ <= radius.  Returned as block CSR over
        basis-atom rows: (rowptr int64[N+1], col int32[nnzb]), columns sorted.
        """
        key = ("w", radius)
        if key in self._bsr_cache:
            return self._bsr_cache[key]
        I, J = _pairs_within(self.positions, radius, include_self=True, both=True)
        rowptr = np.zeros(self.natoms + 1, dtype=np.int64)
        np.add.at(rowptr, I + 1, 1)
        rowptr = np.cumsum(rowptr)
        out = (rowptr, J.astype(np.int32))
        self._bsr_cache[key] = out
        return out

    def w_mask(self, radius: float = W_RADIUS) -> np.ndarray:
        """Dense boolean (m, n) mask of the W pattern (for small systems)."""
        rowptr, col = self.w_pattern(radius)
        blk = np.zeros((self.natoms, self.natoms), dtype=bool)
        rows = np.repeat(np.arange(self.natoms), np.diff(rowptr))
        blk[rows, col] = True
        return np.kron(blk, np.ones((ORB_PER_ATOM, OCC_PER_ATOM), dtype=bool))

    # ---------------------------------------------------------------- W0
    def W0_dense(self) -> np.ndarray:
        """Dense initial guess, (m, n) Fortran-ordered (each orbital contiguous)."""
        rng = np.random.Generator(np.random.PCG64(self.seed + W0_SEED_OFFSET))
        wt = rng.normal(0.0, 1.0 / math.sqrt(self.m), size=(self.n, self.m))
        return wt.T  # F-contiguous view of the (n, m) C array

    def W0_local(self, radius: float = W_RADIUS) -> np.ndarray:
        """Localised initial guess: same draws, kept on the pattern, sigma_j = 1/sqrt(nnz_j)."""
        W = np.array(self.W0_dense(), order="F")
        mask = self.w_mask(radius)
        nnz = mask.sum(axis=0)
        W *= mask
        W *= np.sqrt(self.m / nnz)[None, :]
        return W

    def W0_bsr_values(self, radius: float = W_RADIUS) -> np.ndarray:
        """Localised W0 as 8x2 block values in w_pattern order, (nnzb, 8, 2) row-major.

        Built without forming the dense m x n matrix, so it works at any size;
        equals W0_local() restricted to the pattern.
        """
        rowptr, col = self.w_pattern(radius)
        rng = np.random.Generator(np.random.PCG64(self.seed + W0_SEED_OFFSET))
        m, n, N = self.m, self.n, self.natoms
        # identical draws to W0_dense: (n, m) C order, drawn in slabs to bound memory
        nnzb_col = np.bincount(col, minlength=N)            # blocks per host atom J
        nnz_orb = nnzb_col * ORB_PER_ATOM                    # entries per orbital column
        factor = np.repeat(np.sqrt(m / nnz_orb), OCC_PER_ATOM)   # per orbital j
        sigma = 1.0 / math.sqrt(m)
        vals = np.empty((col.shape[0], ORB_PER_ATOM, OCC_PER_ATOM))
        rows = np.repeat(np.arange(N), np.diff(rowptr))
        # group blocks by host atom J so each slab of orbitals is drawn once
        order_by_J = np.argsort(col, kind="stable")
        J_sorted = col[order_by_J]
        starts = np.searchsorted(J_sorted, np.arange(N))
        ends = np.searchsorted(J_sorted, np.arange(N), side="right")
        for J in range(N):
            slab = rng.normal(0.0, sigma, size=(OCC_PER_ATOM, m))   # orbitals 2J, 2J+1
            slab *= factor[OCC_PER_ATOM * J:OCC_PER_ATOM * (J + 1)][:, None]
            for b in order_by_J[starts[J]:ends[J]]:
                I = rows[b]
                vals[b] = slab[:, I * ORB_PER_ATOM:(I + 1) * ORB_PER_ATOM].T
        return vals


def _pairs_within(pos: np.ndarray, cutoff: float, include_self: bool, both: bool):
    """All (I, J) with |r_I - r_J| <= cutoff, lexicographically sorted.

    A k-d tree proposes candidates within a slightly larger radius; the
    decision itself is the elementwise test dx*dx + dy*dy + dz*dz <= cutoff^2.
    """
    from scipy.spatial import cKDTree

    cand = cKDTree(pos).query_pairs(cutoff * (1.0 + 1e-9) + 1e-12, output_type="ndarray")
    cand = cand.astype(np.int64)
    if cand.size == 0:
        cand = np.zeros((0, 2), dtype=np.int64)
    d = pos[cand[:, 0]] - pos[cand[:, 1]]
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
    cand = cand[r2 <= cutoff * cutoff]
    a = np.minimum(cand[:, 0], cand[:, 1])
    b = np.maximum(cand[:, 0], cand[:, 1])
    Is, Js = [a], [b]
    if both:
        Is.append(b)
        Js.append(a)
    if include_self:
        idx = np.arange(pos.shape[0], dtype=np.int64)
        Is.append(idx)
        Js.append(idx)
    I = np.concatenate(Is)
    J = np.concatenate(Js)
    order = np.lexsort((J, I))
    return I[order], J[order]


def _assemble_dense(N, onsite, pairs, pair_blocks):
    b = ORB_PER_ATOM
    A = np.zeros((N * b, N * b))
    for I in range(N):
        A[I * b:(I + 1) * b, I * b:(I + 1) * b] = onsite[I]
    for (I, J), blk in zip(pairs, pair_blocks):
        A[I * b:(I + 1) * b, J * b:(J + 1) * b] = blk
        A[J * b:(J + 1) * b, I * b:(I + 1) * b] = blk.T
    return A


def grid_positions(nx: int, ny: int, nz: int, natoms: int | None = None) -> np.ndarray:
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    grid = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * GRID_SPACING
    return grid if natoms is None else grid[:natoms]


def make_system(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0,
                natoms: int | None = None) -> System:
    """Generate the system on an nx x ny x nz grid (first `natoms` sites if given)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    base = grid_positions(nx, ny, nz, natoms)
    N = base.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = base + rng.uniform(-JITTER, JITTER, size=(N, 3))
    onsite_diag = ONSITE[None, :] + rng.normal(0.0, ONSITE_SIGMA, size=(N, ORB_PER_ATOM))
    onsite = np.zeros((N, ORB_PER_ATOM, ORB_PER_ATOM))
    idx = np.arange(ORB_PER_ATOM)
    onsite[:, idx, idx] = onsite_diag
    I, J = _pairs_within(pos, HS_CUTOFF, include_self=False, both=False)
    pairs = np.stack([I, J], axis=1)
    dv = pos[I] - pos[J]
    r = np.sqrt(dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1] + dv[:, 2] * dv[:, 2])
    R = rng.standard_normal(size=(pairs.shape[0], ORB_PER_ATOM, ORB_PER_ATOM))
    B = rng.uniform(-1.0, 1.0, size=(pairs.shape[0], ORB_PER_ATOM, ORB_PER_ATOM)) / ORB_PER_ATOM
    H_pair = (0.8 * np.exp(-r / 1.5))[:, None, None] * R
    S_pair = (0.15 * np.exp(-r / 1.2))[:, None, None] * B
    return System(seed=seed, positions=pos, onsite_H=onsite, pairs=pairs, pair_r=r,
                  H_pair=H_pair, S_pair=S_pair)


MD_SEED_OFFSET = 3 * 10 ** 6


def make_md_system(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 0, t: float = 0.0,
                   step: float = 0.1) -> System:
    """Snapshot t of a straight-line MD trajectory of the make_system geometry
    (velocity N(0,1)^3 per atom, `step` Angstrom per unit of t), with pair
    blocks keyed by (seed, I, J) so that H and S follow the positions smoothly."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    base = grid_positions(nx, ny, nz)
    N = base.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = base + rng.uniform(-JITTER, JITTER, size=(N, 3))
    onsite_diag = ONSITE[None, :] + rng.normal(0.0, ONSITE_SIGMA, size=(N, ORB_PER_ATOM))
    vel = np.random.Generator(np.random.PCG64(seed + MD_SEED_OFFSET)).standard_normal((N, 3))
    pos = pos + (t * step) * vel
    onsite = np.zeros((N, ORB_PER_ATOM, ORB_PER_ATOM))
    idx = np.arange(ORB_PER_ATOM)
    onsite[:, idx, idx] = onsite_diag
    I, J = _pairs_within(pos, HS_CUTOFF, include_self=False, both=False)
    pairs = np.stack([I, J], axis=1)
    dv = pos[I] - pos[J]
    r = np.sqrt(dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1] + dv[:, 2] * dv[:, 2])
    R = np.empty((pairs.shape[0], ORB_PER_ATOM, ORB_PER_ATOM))
    B = np.empty_like(R)
    for p, (a, b) in enumerate(pairs):
        prng = np.random.Generator(np.random.PCG64([seed, int(a), int(b)]))
        R[p] = prng.standard_normal((ORB_PER_ATOM, ORB_PER_ATOM))
        B[p] = prng.uniform(-1.0, 1.0, size=(ORB_PER_ATOM, ORB_PER_ATOM)) / ORB_PER_ATOM
    H_pair = (0.8 * np.exp(-r / 1.5))[:, None, None] * R
    S_pair = (0.15 * np.exp(-r / 1.2))[:, None, None] * B
    return System(seed=seed, positions=pos, onsite_H=onsite, pairs=pairs, pair_r=r,
                  H_pair=H_pair, S_pair=S_pair)


def make_dense_gapped(m: int, n: int, seed: int):
    """Generic dense inputs of any size (the ragged-size cases, m not a multiple
    of the block or tile sizes): H = Q diag(lam) Q^T with n eigenvalues
    U(-6, -3) and m - n eigenvalues U(3, 8) eV, Q the Q factor of an N(0,1)
    matrix; S = I + (A + A^T)/2 with A ~ N(0, 0.15/m) (strictly diagonally
    dominant, SPD); T = I + (B B^T)/m with B ~ N(0,1) (SPD); W0 ~ N(0, 1/sqrt(m)).
    One PCG64 stream seeded with `seed`, drawn in that order.  Returns
    (H, S, T, W0) as Fortran-ordered arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    lam = np.concatenate([rng.uniform(-6.0, -3.0, n), rng.uniform(3.0, 8.0, m - n)])
    H = (Q * lam) @ Q.T
    H = 0.5 * (H + H.T)
    A = rng.normal(0.0, 0.15 / m, size=(m, m))
    S = np.eye(m) + 0.5 * (A + A.T)
    B = rng.standard_normal((m, m))
    T = np.eye(m) + (B @ B.T) / m
    W0 = rng.normal(0.0, 1.0 / math.sqrt(m), size=(m, n))
    return tuple(np.asfortranarray(x) for x in (H, S, T, W0))


def batch_sizes(count: int, seed: int, lo: int = 32, hi: int = 384) -> np.ndarray:
    """Atom counts for a batch of uneven systems: round(exp(U(ln lo, ln hi)))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def make_batch_system(natoms: int, seed: int) -> System:
    side = int(math.ceil(round(natoms ** (1.0 / 3.0), 9)))
    while side ** 3 < natoms:
        side += 1
    return make_system(side, side, side, seed=seed, natoms=natoms)


def perturb_pairs(sys: System, seq_seed: int, step: int, sigma: float = 1e-3) -> System:
    """SCF-like perturbation of H on its existing nonzeros, symmetric by construction.

    Adds N(0, sigma) to every stored onsite-diagonal entry and to every entry of
    every stored pair block (the transpose block follows).  Draws come from a
    PCG64 stream seeded with (seq_seed, step).
    """
    rng = np.random.Generator(np.random.PCG64([seq_seed, step]))
    N = sys.natoms
    d_on = rng.normal(0.0, sigma, size=(N, ORB_PER_ATOM))
    d_pair = rng.normal(0.0, sigma, size=sys.H_pair.shape)
    onsite = sys.onsite_H.copy()
    idx = np.arange(ORB_PER_ATOM)
    onsite[:, idx, idx] += d_on
    return System(seed=sys.seed, positions=sys.positions, onsite_H=onsite, pairs=sys.pairs,
                  pair_r=sys.pair_r, H_pair=sys.H_pair + d_pair, S_pair=sys.S_pair)
