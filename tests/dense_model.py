"""Dense textbook construction of the Holstein Hamiltonian for tiny systems.

Used only by the tests as an independent check of the oracle: the operator is
assembled from Kronecker products of single-site ladder matrices (Eq. holstein),
not from the move rules the oracle and the kernels use.
"""
import numpy as np


def ladder(K):
    """annihilation operator on {|0>..|K>}: a|n> = sqrt(n)|n-1>"""
    return np.diag(np.sqrt(np.arange(1, K + 1, dtype=np.float64)), 1)


def site_operator(j, op, dims):
    out = np.eye(1)
    for i, d in enumerate(dims):
        out = np.kron(out, op if i == j else np.eye(d))
    return out


def dense_holstein(hop, eps, omega, g, caps):
    """H on C^N (x) (x)_j C^{K_j+1}; basis index = s * D + sum_j n_j stride_j."""
    N = len(eps)
    dims = [int(K) + 1 for K in caps]
    D = int(np.prod(dims))
    hexc = np.diag(np.asarray(eps, dtype=np.float64)) + np.asarray(hop, dtype=np.float64)
    H = np.kron(hexc, np.eye(D))
    hph = np.zeros((D, D))
    for j in range(N):
        a = ladder(dims[j] - 1)
        hph += omega[j] * site_operator(j, a.T @ a, dims)
    H += np.kron(np.eye(N), hph)
    for s in range(N):
        if g[s] == 0.0:
            continue
        a = ladder(dims[s] - 1)
        P = np.zeros((N, N))
        P[s, s] = 1.0
        H += g[s] * np.kron(P, site_operator(s, a + a.T, dims))
    strides = [int(np.prod(dims[j + 1:])) for j in range(N)]
    return H, D, strides


def dense_index(tuples, D, strides):
    t = np.asarray(tuples)
    return t[:, 0] * D + t[:, 1:] @ np.asarray(strides)


def ring_hop(N, J):
    h = np.zeros((N, N))
    for a in range(N):
        b = (a + 1) % N
        if a != b:
            h[a, b] = h[b, a] = J
    return h


def propagator(H):
    w, V = np.linalg.eigh(H)
    return lambda t, psi: V @ (np.exp(-1j * w * t) * (V.conj().T @ psi))
