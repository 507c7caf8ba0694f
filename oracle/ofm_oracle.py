"""Plain FP64 CPU oracle of the overlapping fragments method (OFM).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path.

What it computes, step by step, in the paper's order (Vukmirovic & Wang,
"Overlapping fragments method for electronic structure calculation of large
systems", Sec. II):

1. The single-particle Hamiltonian of Eq. 1 on a periodic real-space grid:
   H = -1/2 Laplacian + V (atomic units), the Laplacian being the 7-point
   finite difference  (sum of the 6 neighbours - 6 phi(r)) / h^2.
2. Fragment basis (Sec. II, "calculation of basis wave functions"): the lowest
   n_a eigenpairs of the fragment Hamiltonian, read here as the principal
   submatrix of the global H on the fragment's box (zero outside the box,
   periodic wrap kept in a dimension the box spans completely).  States are
   unit-norm in the plain Euclidean grid sum, ascending in energy, with the
   sign gauge "largest |component| positive, ties to the lowest index".
3. H phi_b for every fragment state, with the whole-system H (Sec. II),
   evaluated on the box dilated by one point, where it can be non-zero.
4. For every pair of fragments whose boxes interact (box a meets the dilated
   box of b) the blocks S_ab = <phi_a|phi_b> and H_ab = <phi_a|H|phi_b>
   (Sec. II, the transfer integrals and overlaps), computed here from their
   definition with zero-extended whole-grid vectors.  The block a<b is kept
   as computed, the block b>a is its transpose, and a diagonal block is
   symmetrised as (X + X^T)/2.
5. The generalized eigenproblem sum_mn (H - E S) C = 0 of Eq. 2 on the dense
   assembled matrices (LAPACK through scipy.linalg.eigh, as the paper uses
   standard LAPACK routines), and the eigenvalues inside an energy window.
6. Variants of Sec. III: the distance cutoff on the pair list ("Choice of the
   distance cutoff"), and, for a basis of fragment HOMOs ("Choice of the
   number of basis states per fragment"), e_i = <i|H|i> and the first gap of
   the spectrum above it.

Readings of the paper where it is silent are listed in the repository's
design notes (fragment Hamiltonian = principal submatrix; the H_ab sum runs
over the one-point halo where H phi_b is non-zero; plain Euclidean inner
products; pair criterion = exact geometric overlap of box a with the dilated
box b).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg

DENSE_EIGH_MAX = 4096


# ---------------------------------------------------------------- geometry --

def box_axes(grid, off, ext):
    """Per-dimension global coordinates of box off + [0, ext) (mod n)."""
    return [np.mod(off[d] + np.arange(ext[d]), grid.n[d]) for d in range(3)]


def box_indices(grid, off, ext):
    """Global linear indices (x fastest) of the box points, in box order
    (x fastest, then y, then z)."""
    nx, ny, _ = grid.n
    gx, gy, gz = box_axes(grid, off, ext)
    return (gz[:, None, None] * (nx * ny) + gy[None, :, None] * nx
            + gx[None, None, :]).ravel()


def dilated_box(grid, frag):
    """Box grown by one point on each side in every dimension the box does
    not already span completely (Sec. II: H phi reaches one point beyond the
    box through the finite-difference stencil)."""
    off, ext = [], []
    for d in range(3):
        if frag.ext[d] < grid.n[d]:
            off.append(frag.off[d] - 1)
            ext.append(frag.ext[d] + 2)
        else:
            off.append(frag.off[d])
            ext.append(frag.ext[d])
    return tuple(off), tuple(ext)


# ------------------------------------------------------------- Hamiltonian --

def hamiltonian(grid, V):
    """Global H of Eq. 1 as a sparse matrix: diagonal 3/h^2 + V(r), and
    -1/(2 h^2) between each point and each of its 6 periodic neighbours."""
    nx, ny, nz = grid.n
    N = nx * ny * nz
    h2 = grid.h * grid.h
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = (k * ny * nx + j * nx + i).ravel()
    rows = [idx]
    cols = [idx]
    vals = [np.full(N, 3.0 / h2) + np.asarray(V, dtype=np.float64).ravel()]
    for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        nb = (np.mod(k + dk, nz) * ny * nx + np.mod(j + dj, ny) * nx + np.mod(i + di, nx)).ravel()
        rows.append(idx)
        cols.append(nb)
        vals.append(np.full(N, -0.5 / h2))
    H = scipy.sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(N, N)).tocsr()
    H.sum_duplicates()
    return H


def fragment_hamiltonian(H, grid, frag):
    """Principal submatrix of H on the fragment box (box order)."""
    idx = box_indices(grid, frag.off, frag.ext)
    return H[idx][:, idx]


def gauge_fix(Phi):
    """Sign of each column chosen so that its largest-magnitude entry is
    positive (ties: the lowest index, which argmax returns)."""
    Phi = np.array(Phi, dtype=np.float64, copy=True)
    for c in range(Phi.shape[1]):
        i = int(np.argmax(np.abs(Phi[:, c])))
        if Phi[i, c] < 0:
            Phi[:, c] = -Phi[:, c]
    return Phi


def fragment_eigs(H, grid, frag, n_extra=0):
    """Lowest n_a (+ n_extra) eigenpairs of the fragment Hamiltonian.

    Dense LAPACK eigh for boxes up to DENSE_EIGH_MAX points; above that,
    shift-invert Lanczos (ARPACK) with the shift below the whole spectrum.
    Returns (eps ascending, Phi with unit-norm columns in box order)."""
    Hf = fragment_hamiltonian(H, grid, frag)
    P = Hf.shape[0]
    k = frag.n_states + n_extra
    if P <= DENSE_EIGH_MAX:
        w, U = np.linalg.eigh(Hf.toarray())
        w, U = w[:k], U[:, :k]
    else:
        sigma = float(Hf.diagonal().min()) - 4.0 / grid.h ** 2
        w, U = scipy.sparse.linalg.eigsh(Hf.tocsc(), k=k, sigma=sigma, which="LM",
                                         tol=1e-14, maxiter=100000)
        order = np.argsort(w)
        w, U = w[order], U[:, order]
    U = U / np.linalg.norm(U, axis=0)
    return w, gauge_fix(U)


# ------------------------------------------------------------- H apply ------

def zero_extend(grid, frag, Phi):
    """Fragment states as whole-grid vectors, zero outside the box."""
    idx = box_indices(grid, frag.off, frag.ext)
    n = Phi.shape[1]
    rows = np.repeat(idx, n)
    cols = np.tile(np.arange(n), len(idx))
    return scipy.sparse.csr_matrix((np.asarray(Phi, dtype=np.float64).ravel(), (rows, cols)),
                                   shape=(grid.npoints, n))


def apply_h(H, grid, frag, Phi):
    """H phi_b with the whole-system H (Sec. II), returned on the dilated
    box in dilated-box order (x fastest)."""
    HPhi = (H @ zero_extend(grid, frag, Phi)).toarray()
    doff, dext = dilated_box(grid, frag)
    return HPhi[box_indices(grid, doff, dext)]


# ------------------------------------------------------------- pairs --------

def boxes_meet(grid, offa, exta, offb, extb):
    """True when two periodic boxes share a grid point: boxes are products
    of per-dimension point sets, so they meet when every dimension does."""
    for d in range(3):
        sa = set(np.mod(offa[d] + np.arange(exta[d]), grid.n[d]).tolist())
        sb = set(np.mod(offb[d] + np.arange(extb[d]), grid.n[d]).tolist())
        if not (sa & sb):
            return False
    return True


def pair_list(grid, frags):
    """Unordered pairs a <= b whose blocks are structurally non-zero: box a
    meets the dilated box of b (then H_ab may be non-zero; S_ab may still be
    zero when only the one-point halo is shared)."""
    dil = [dilated_box(grid, f) for f in frags]
    out = []
    for a, fa in enumerate(frags):
        for b in range(a, len(frags)):
            if boxes_meet(grid, fa.off, fa.ext, dil[b][0], dil[b][1]):
                out.append((a, b))
    return out


def fragment_distance(grid, atoms_a, atoms_b):
    """Sec. III.C: the distance between two fragments is the minimal distance
    between an atom of one and an atom of the other (minimum image in the
    periodic box of n[d] * h bohr).  Infinite when either has no atoms."""
    L = [grid.n[d] * grid.h for d in range(3)]
    best = math.inf
    for ra in np.asarray(atoms_a, dtype=np.float64).reshape(-1, 3):
        for rb in np.asarray(atoms_b, dtype=np.float64).reshape(-1, 3):
            s = 0.0
            for d in range(3):
                x = ra[d] - rb[d]
                x -= L[d] * round(x / L[d])
                s += x * x
            best = min(best, math.sqrt(s))
    return best


def cutoff_pairs(grid, frags, atoms, d_cut):
    """Sec. III.C: the pair list restricted to fragments closer than d_cut
    (self pairs always kept); atoms[a] holds fragment a's atom positions."""
    return [(a, b) for (a, b) in pair_list(grid, frags)
            if a == b or fragment_distance(grid, atoms[a], atoms[b]) < d_cut]


def overlap_points(grid, offa, exta, offb, extb):
    """Number of grid points shared by two periodic boxes."""
    cnt = 1
    for d in range(3):
        sa = set(np.mod(offa[d] + np.arange(exta[d]), grid.n[d]).tolist())
        sb = set(np.mod(offb[d] + np.arange(extb[d]), grid.n[d]).tolist())
        cnt *= len(sa & sb)
    return cnt


def pair_flops(grid, frags, pairs):
    """Algorithmic flop count of the pair blocks: for a <= b,
    2 n_a n_b (|B_a ∩ B_b| + |B_a ∩ B_b^+|)."""
    F = 0
    for a, b in pairs:
        fa, fb = frags[a], frags[b]
        doff, dext = dilated_box(grid, fb)
        k_s = overlap_points(grid, fa.off, fa.ext, fb.off, fb.ext)
        k_h = overlap_points(grid, fa.off, fa.ext, doff, dext)
        F += 2 * fa.n_states * fb.n_states * (k_s + k_h)
    return F


# ------------------------------------------------------------- blocks -------

def pair_block(H, grid, fa, Phia, fb, Phib):
    """(H_ab, S_ab) = (<phi_a|H|phi_b>, <phi_a|phi_b>) from zero-extended
    whole-grid vectors (Sec. II)."""
    Ea = zero_extend(grid, fa, Phia)
    Eb = zero_extend(grid, fb, Phib)
    S = (Ea.T @ Eb).toarray()
    Hb = (Ea.T @ (H @ Eb)).toarray()
    return Hb, S


def pair_blocks(H, grid, frags, Phis, pairs=None, symmetrise=True):
    """Blocks for every pair a <= b; diagonal blocks symmetrised."""
    if pairs is None:
        pairs = pair_list(grid, frags)
    out = {}
    for a, b in pairs:
        Hab, Sab = pair_block(H, grid, frags[a], Phis[a], frags[b], Phis[b])
        if a == b and symmetrise:
            Hab = 0.5 * (Hab + Hab.T)
            Sab = 0.5 * (Sab + Sab.T)
        out[(a, b)] = (Hab, Sab)
    return out


def assemble_dense(frags, blocks):
    """Dense H and S in basis order (fragment-major, states ascending); the
    block b>a is the transpose of the computed block a<b."""
    starts = np.concatenate([[0], np.cumsum([f.n_states for f in frags])])
    n = int(starts[-1])
    Hd = np.zeros((n, n))
    Sd = np.zeros((n, n))
    for (a, b), (Hab, Sab) in blocks.items():
        ra = slice(starts[a], starts[a + 1])
        rb = slice(starts[b], starts[b + 1])
        Hd[ra, rb] = Hab
        Sd[ra, rb] = Sab
        if a != b:
            Hd[rb, ra] = Hab.T
            Sd[rb, ra] = Sab.T
    return Hd, Sd


# ------------------------------------------------------------- Eq. 2 --------

def generalized_eigs(Hd, Sd):
    """All eigenvalues of sum_mn (H - E S) C = 0 (Eq. 2), ascending, through
    LAPACK's Cholesky-based symmetric-definite solver."""
    return scipy.linalg.eigh(Hd, Sd, eigvals_only=True)


def generalized_eigs_jacobi(Hd, Sd, sweeps=60, tol=1e-15):
    """Second opinion for small problems, written out by hand: Cholesky
    S = L L^T, A = L^-1 H L^-T, cyclic Jacobi rotations on A."""
    n = Hd.shape[0]
    L = np.zeros((n, n))
    for j in range(n):
        s = Sd[j, j] - L[j, :j] @ L[j, :j]
        if s <= 0:
            raise np.linalg.LinAlgError("S is not positive definite")
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (Sd[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]
    Linv = np.linalg.inv(L)
    A = Linv @ Hd @ Linv.T
    A = 0.5 * (A + A.T)
    for _ in range(sweeps):
        off = np.sqrt(np.sum(np.tril(A, -1) ** 2))
        if off <= tol * max(1.0, np.abs(np.diag(A)).max()):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if abs(A[p, q]) < 1e-300:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * A[p, q])
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                Ap = A[:, p].copy()
                Aq = A[:, q].copy()
                A[:, p] = c * Ap - s * Aq
                A[:, q] = s * Ap + c * Aq
                Ap = A[p, :].copy()
                Aq = A[q, :].copy()
                A[p, :] = c * Ap - s * Aq
                A[q, :] = s * Ap + c * Aq
    return np.sort(np.diag(A))


def window_bounds(E, rule):
    """Energy window [E_lo, E_hi] from a reference spectrum E (ascending)
    and a window rule (reading of the paper's gap procedure, Sec. III.B,
    for a synthetic potential with no electron count: one occupied level
    per well)."""
    if rule.kind == "from_lowest":
        return float(E[0]), float(E[0] + rule.width)
    if rule.kind == "above_gap":
        lo = float(E[rule.n_occ])
        return lo, lo + rule.width
    if rule.kind == "around_gap":
        return float(E[rule.n_occ - 1] - rule.width), float(E[rule.n_occ] + rule.width)
    raise ValueError(rule.kind)


def window_eigs(Hd, Sd, E_lo, E_hi):
    """Eigenvalues of Eq. 2 inside [E_lo, E_hi] (inclusive), ascending."""
    E = generalized_eigs(Hd, Sd)
    return E[(E >= E_lo) & (E <= E_hi)]


def window_vectors(Hd, Sd, E_lo, E_hi):
    """Eigenpairs of Eq. 2 inside [E_lo, E_hi] (inclusive): eigenvalues
    ascending and the coefficient vectors C (columns, S-orthonormal:
    C^T S C = I), from LAPACK's symmetric-definite solver."""
    E, C = scipy.linalg.eigh(Hd, Sd)
    keep = (E >= E_lo) & (E <= E_hi)
    return E[keep], C[:, keep]


# ------------------------------------------------------------- pipeline -----

def homo_expectations(H, grid, frags, Phis):
    """Sec. III (occupation with a HOMO basis): e_a = <i|H|i> with the
    whole-system H, |i> the highest basis state of fragment a."""
    out = []
    for f, P in zip(frags, Phis):
        v = np.asarray(zero_extend(grid, f, P[:, -1:]).todense()).ravel()
        out.append(float(v @ (H @ v)))
    return out


def first_gap(E, e_ref, gap_min):
    """Sec. III: the first gap in the spectrum above e_ref, read as the first
    spacing wider than gap_min between consecutive eigenvalues, starting from
    the largest eigenvalue <= e_ref.  Returns (E_homo, E_lumo, n_occ) with
    n_occ the number of eigenvalues <= E_homo."""
    E = np.sort(np.asarray(E, dtype=np.float64))
    k = max(int(np.sum(E <= e_ref)) - 1, 0)
    for i in range(k, len(E) - 1):
        if E[i + 1] - E[i] > gap_min:
            return float(E[i]), float(E[i + 1]), i + 1
    raise ValueError("no spacing wider than gap_min at or above e_ref")


def run_ofm(workload, Phis=None, pairs=None):
    """Whole method on one workload: fragment eigensolves (unless states are
    given), H phi, pair blocks, dense assembly and the full spectrum of
    Eq. 2.  Returns a dict of every intermediate."""
    grid, frags = workload.grid, workload.frags
    H = hamiltonian(grid, workload.V)
    eps = None
    if Phis is None:
        eps, Phis = [], []
        for f in frags:
            w, U = fragment_eigs(H, grid, f)
            eps.append(w)
            Phis.append(U)
    if pairs is None:
        pairs = pair_list(grid, frags)
    blocks = pair_blocks(H, grid, frags, Phis, pairs)
    Hd, Sd = assemble_dense(frags, blocks)
    E = generalized_eigs(Hd, Sd)
    return dict(H=H, eps=eps, Phis=Phis, pairs=pairs, blocks=blocks, Hd=Hd, Sd=Sd, E=E)
