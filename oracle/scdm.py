"""FP64 oracle for SCDM localisation with the s'-MTACE pre-selection
(arXiv:2110.07670 Sections 2.4-2.5).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the bench's
CPU-baseline leg may use it.  It shares nothing with the CUDA library; the
real-space orbitals come from this package's own transforms (to_real), and
every step below is written out plainly in numpy, in the paper's order:

1. electron density rho(r) = sum_i psi_i(r)^2 and its gradient
   grad rho = 2 sum_i psi_i grad psi_i, where grad psi_i is the exact
   derivative of the plane-wave expansion (coefficients i G c_i(G));
2. pre-selection (Section 2.5): grid point r is a candidate when
   rho(r) > <rho> and |grad rho(r)| < <|grad rho|> (averages over all grid
   points); without pre-selection every grid point is a candidate;
3. rank-revealing QR with column pivoting of Psi^* restricted to the
   candidate columns (Section 2.4): Householder QR, at each step the column
   of largest remaining norm (norms recomputed from the trailing block, ties
   to the lowest index) -- the first n_occ pivots C are kept;
4. the selected columns of the density matrix Gamma = Psi Psi^*,
   phi~_k(r) = sum_i psi_i(r) psi_i(r_{C_k}), orthonormalised symmetrically
   (Loewdin): Phi = (V V^T)^{-1/2} V Psi with V[k][i] = psi_i(r_{C_k}).

Readings (also in the design notes): one electron per orbital in rho (a
constant factor changes neither comparison); |grad rho| is the Euclidean norm;
the Loewdin orthonormalisation of the selected columns; a best residual
norm^2 at or below 1e-10 of the largest column norm^2 is rank deficiency.
"""
import numpy as np

from . import half_sphere, to_real


def reciprocal_rows(cell):
    """b_j (rows) with a_i . b_j = 2 pi delta_ij for the lattice vectors a_i (rows of cell)."""
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    return 2.0 * np.pi * np.linalg.inv(a).T


def density_and_gradient(psi, cell, grid, ecut):
    """rho [N] and grad rho [3][N] on the grid (box order i0, i1, i2)."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    m = half_sphere(cell, ecut)
    G = m.astype(np.float64) @ reciprocal_rows(cell)  # [n_pw_half][3]
    phi = to_real(psi, cell, grid, ecut).reshape(len(psi), -1)
    rho = (phi * phi).sum(0)
    grad = np.zeros((3, phi.shape[1]))
    for d in range(3):
        dphi = to_real(psi * (1j * G[:, d])[None, :], cell, grid, ecut).reshape(len(psi), -1)
        grad[d] = 2.0 * (phi * dphi).sum(0)
    return rho, grad


def preselect(rho, grad):
    """Ascending indices of the grid points with rho > <rho> and |grad rho| < <|grad rho|>."""
    gn = np.sqrt((grad * grad).sum(0))
    return np.nonzero((rho > rho.mean()) & (gn < gn.mean()))[0]


def qrcp_pivots(A, k):
    """First k pivot columns of Householder QR with column pivoting of A
    (rows x columns), each step taking the column of largest trailing norm.
    Rank deficient (ValueError) when that norm^2 is not above 1e-10 times the
    largest column norm^2 of A: fewer than k independent columns beyond
    rounding.  Where 1e-10 comes from: columns that are dependent in exact
    arithmetic keep a trailing norm^2 at the level of their inputs' rounding,
    u^2 of the largest column's -- about 4e-15 for orbitals stored in single
    precision (u = 2^-24), 1e-32 for double -- plus the evaluation's own
    error (at most m 2^-53 in FP64 or 2^-44 in float-float per entry, m <=
    2048 rows, so below 1e-22 in norm^2).  A column whose independent part is
    above 1e-5 of the largest (norm^2 above 1e-10) is therefore told apart
    from a dependent one by four orders in either precision."""
    R = np.array(A, dtype=np.float64)
    nr, nc = R.shape
    perm = np.arange(nc)
    ref = float((R * R).sum(0).max())
    for s in range(k):
        norms = (R[s:, s:] ** 2).sum(0)
        j = s + int(np.argmax(norms))  # argmax returns the first of equal maxima
        if not norms[j - s] > 1e-10 * ref:
            raise ValueError("rank deficient: fewer than %d independent columns" % k)
        R[:, [s, j]] = R[:, [j, s]]
        perm[[s, j]] = perm[[j, s]]
        if s == nr - 1:
            continue
        x = R[s:, s].copy()
        alpha = -np.copysign(np.linalg.norm(x), x[0])
        v = x
        v[0] -= alpha
        v /= np.linalg.norm(v)
        R[s:, s:] -= 2.0 * np.outer(v, v @ R[s:, s:])
    return perm[:k]


def scdm(psi, cell, grid, ecut, use_preselect=True):
    """dict(phi_G, pivots, O, candidates): localised orbitals phi_G = O psi_G
    (same half-sphere layout), the n_occ pivot grid points, the orthogonal
    n_occ x n_occ rotation O and the candidate grid points."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    n = len(psi)
    phi = to_real(psi, cell, grid, ecut).reshape(n, -1)
    if use_preselect:
        rho, grad = density_and_gradient(psi, cell, grid, ecut)
        cand = preselect(rho, grad)
    else:
        cand = np.arange(phi.shape[1])
    if len(cand) < n:
        raise ValueError("pre-selection kept %d grid points for %d orbitals" % (len(cand), n))
    piv = cand[qrcp_pivots(phi[:, cand], n)]
    V = phi[:, piv].T  # V[k][i] = psi_i(r_{C_k})
    w, E = np.linalg.eigh(V @ V.T)
    O = (E * w ** -0.5) @ E.T @ V
    return dict(phi_G=O @ psi, pivots=piv, O=O, candidates=cand)
