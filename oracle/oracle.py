"""Plain CPU FP64 oracle for the binned harmonic 3PCF estimator.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).  The
library never imports this module.

Definitions followed (arXiv:2408.16847, section 3.1):

* eq. Xm.binned: for each pivot i, X_m(theta^a; nu_i) sums w_j x_j e^{i m phi_j}
  over the neighbours j in radial bin a.  The oracle keeps the unnormalised sum
  with the conjugate phase convention  a_m^k(i) = sum_j w_j d_j e^{-i m phi_ij}
  (phi_ij = position angle of j about i, from local north through east).
* eq. zetamEst / zetamEst2: zeta_m(theta1, theta2) averages over pivots p the
  field value w_p x_p times the outer product X_m(theta1) X_{-m}(theta2).  With
  the convention above X_{-m} = conj(X_m) for a real field, so
      S_m(k1,k2) = sum_i w_i d_i a_m^{k1}(i) conj(a_m^{k2}(i)).
  (The printed eq. zetamEst writes w_j x_j inside the pivot sum; eq. zetamEst2
  writes w_p x_p, which is the reading used.)
* normalisation (three readings, selected by ``norm``):
    "R3"  zeta = S / D with D the same estimator run with d = 1 and m = 0,
          D(k1,k2) = sum_i w_i W^{k1}(i) W^{k2}(i)          (default)
    "R2"  per pivot and bin, X = a / W (the "average over all points in that bin"
          of the binning-scheme figure), then divided by sum_i w_i
    "R1"  per pivot, X = a / sum_{j in any bin} w_j (the prefactor of eq. Xm.binned),
          then divided by sum_i w_i (the prefactor of eq. zetamEst).
* self pairs (section 3.4): the j = k term of X_m (x) X_{-m} is kept by default
  ("keep"); "subtract" removes sum_i w_i d_i sum_j (w_j d_j)^2 Theta_k(ij) from
  every S_m(k,k) (and the d = 1 version from D(k,k)).

Bins are compared by chord c = |n_j - n_i| against c_e = 2 sin(theta_e / 2) in FP64,
half-open [theta_k, theta_{k+1}).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (in-tree, plain C + OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    out = os.path.join(_HERE, "_oracle.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.orc_pix2vec_ring.argtypes = [_i64, _i64, _p, _p]
            lib.orc_pix2vec_all.argtypes = [_i64, _p]
            lib.orc_pix2vec_one.argtypes = [_i64, _i64, _p]
            lib.orc_moments.argtypes = [_i64, _p, _p, _p, _i64, _p, ctypes.c_int, _p, ctypes.c_int,
                                        _p, _p, _p, _p, _p, _p]
            lib.orc_moments.restype = ctypes.c_int
            lib.orc_neighbor_legs.argtypes = [_i64, _p, _p, _p, _i64, _p, _p, ctypes.c_int, _p,
                                              ctypes.c_int, _i64, _p, _p]
            lib.orc_neighbor_legs.restype = ctypes.c_int
            lib.orc_pair_counts.argtypes = [_i64, _p, _i64, _p, ctypes.c_int, _p, _p]
            lib.orc_pair_counts.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64a(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


# ----------------------------------------------------------------- geometry

def pix2vec_ring(nside: int, pix=None) -> np.ndarray:
    """HEALPix RING pixel centres (Gorski et al. 2005), float64 (n, 3)."""
    if pix is None:
        out = np.empty((12 * nside * nside, 3))
        _lib().orc_pix2vec_all(nside, out.ctypes.data)
        return out
    pix = _i64a(pix)
    out = np.empty((len(pix), 3))
    _lib().orc_pix2vec_ring(nside, len(pix), pix.ctypes.data, out.ctypes.data)
    return out


def chord_edges(edges_deg) -> np.ndarray:
    """Chord of each angular edge, c = 2 sin(theta / 2), theta in radians (FP64)."""
    th = np.deg2rad(_f64(edges_deg))
    return 2.0 * np.sin(0.5 * th)


# ------------------------------------------------------------------ moments

def moments(xyz, delta, w, edges_deg, m_max: int, pivots=None, psi=None):
    """Per-pivot moments a (npiv, K, M+1) complex, W, Q, QW (npiv, K), and stats.

    ``pivots`` are point indices (default: all points).  ``psi`` rotates each pivot's
    reference direction by psi[t] (phi -> phi - psi).
    """
    xyz = _f64(xyz)
    n = xyz.shape[0]
    delta = _f64(delta)
    w = _f64(w)
    piv = np.arange(n, dtype=np.int64) if pivots is None else _i64a(pivots)
    ce = chord_edges(edges_deg)
    K = len(ce) - 1
    M = int(m_max)
    npiv = len(piv)
    a = np.zeros((npiv, K, M + 1, 2))
    W = np.zeros((npiv, K))
    Q = np.zeros((npiv, K))
    QW = np.zeros((npiv, K))
    st = np.zeros(2)
    ps = None if psi is None else _f64(psi)
    rc = _lib().orc_moments(n, xyz.ctypes.data, delta.ctypes.data, w.ctypes.data, npiv,
                            piv.ctypes.data, K, ce.ctypes.data, M,
                            None if ps is None else ps.ctypes.data,
                            a.ctypes.data, W.ctypes.data, Q.ctypes.data, QW.ctypes.data,
                            st.ctypes.data)
    if rc != 0:
        raise RuntimeError("orc_moments failed (%d)" % rc)
    return dict(a=a[..., 0] + 1j * a[..., 1], W=W, Q=Q, QW=QW, pivots=piv,
                pairs=int(st[0]), min_margin=float(st[1]))


def contract(mom, delta, w, norm: str = "R3", self_pairs: str = "keep"):
    """S, D and zeta from per-pivot moments (eqs. zetamEst / zetamEst2).

    Returns dict with S (M+1, K, K) complex, D (K, K), zeta (M+1, K, K) complex.
    """
    piv = mom["pivots"]
    wi = _f64(w)[piv]
    di = _f64(delta)[piv]
    a, W = mom["a"], mom["W"]
    wd = wi * di
    if norm == "R3":
        S = np.einsum("i,ikm,ilm->mkl", wd, a, np.conj(a))
        D = np.einsum("i,ik,il->kl", wi, W, W)
        if self_pairs == "subtract":
            K = a.shape[1]
            sub = np.einsum("i,ik->k", wd, mom["Q"])
            subd = np.einsum("i,ik->k", wi, mom["QW"])
            S = S.copy()
            D = D.copy()
            S[:, np.arange(K), np.arange(K)] -= sub[None, :]
            D[np.arange(K), np.arange(K)] -= subd
        with np.errstate(divide="ignore", invalid="ignore"):
            zeta = np.where(D[None] != 0, S / np.where(D == 0, 1.0, D)[None], 0.0)
        return dict(S=S, D=D, zeta=zeta)
    if self_pairs != "keep":
        raise ValueError("self-pair subtraction is defined for R3 only")
    if norm == "R2":
        with np.errstate(divide="ignore", invalid="ignore"):
            X = np.where(W[:, :, None] > 0, a / np.where(W > 0, W, 1.0)[:, :, None], 0.0)
    elif norm == "R1":
        tot = W.sum(axis=1)
        with np.errstate(divide="ignore", invalid="ignore"):
            X = np.where(tot[:, None, None] > 0, a / np.where(tot > 0, tot, 1.0)[:, None, None], 0.0)
    else:
        raise ValueError(norm)
    S = np.einsum("i,ikm,ilm->mkl", wd, X, np.conj(X))
    sw = wi.sum()
    zeta = S / sw if sw != 0 else np.zeros_like(S)
    return dict(S=S, D=np.full((a.shape[1], a.shape[1]), sw), zeta=zeta)


def zeta(xyz, delta, w, edges_deg, m_max: int, pivots=None, norm: str = "R3",
         self_pairs: str = "keep", psi=None):
    """The estimator: moments + contraction + normalisation.  Adds 'pairs' and
    'min_margin' (smallest relative chord-to-edge distance among candidate pairs)."""
    mom = moments(xyz, delta, w, edges_deg, m_max, pivots, psi)
    out = contract(mom, delta, w, norm, self_pairs)
    out["pairs"] = mom["pairs"]
    out["min_margin"] = mom["min_margin"]
    out["moments"] = mom
    return out


# ------------------------------------------------------------------ adjoint

def gradient(xyz, delta, w, edges_deg, m_max: int, dL_dzeta, pivots=None, targets=None,
             self_pairs: str = "keep"):
    """dL/d(delta_p) for the targets p, for a real loss L(zeta) of the R3 estimator
    restricted to the pivot set ``pivots``.

    ``dL_dzeta`` (M+1, K, K) complex holds dL/dRe(zeta) + i dL/dIm(zeta).  With
    C = dL_dzeta / D the derivative of the product rule on S is
        w_p sum_{m,k1,k2} Re[conj(C) a^{k1}(p) conj(a^{k2}(p))]                (p a pivot)
      + w_p sum_{i in P, p in nbr(i)} w_i d_i sum_m Re[e^{-i m phi_ip} h_m^{k(ip)}(i)],
        h_m^k(i) = sum_{k'} (conj(C_m(k,k')) + C_m(k',k)) conj(a_m^{k'}(i)),
    plus, for self-pair subtraction, the derivative of the subtracted diagonal.
    """
    xyz = _f64(xyz)
    n = xyz.shape[0]
    delta = _f64(delta)
    w = _f64(w)
    tgt = np.arange(n, dtype=np.int64) if targets is None else _i64a(targets)
    mom = moments(xyz, delta, w, edges_deg, m_max, pivots)
    piv = mom["pivots"]
    res = contract(mom, delta, w, "R3", self_pairs)
    D = res["D"]
    G = np.asarray(dL_dzeta, dtype=np.complex128)
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.where(D[None] != 0, G / np.where(D == 0, 1.0, D)[None], 0.0)
    a = mom["a"]  # (npiv, K, M+1)
    # primary term for targets that are pivots
    pos = np.full(n, -1, dtype=np.int64)
    pos[piv] = np.arange(len(piv))
    grad = np.zeros(len(tgt))
    tp = pos[tgt]
    isp = tp >= 0
    if np.any(isp):
        ap = a[tp[isp]]
        prim = np.einsum("mkl,ikm,ilm->i", np.conj(C), ap, np.conj(ap)).real
        if self_pairs == "subtract":
            K = a.shape[1]
            cdiag = np.conj(C)[:, np.arange(K), np.arange(K)].real.sum(axis=0)  # (K,)
            prim = prim - mom["Q"][tp[isp]] @ cdiag
        grad[isp] += w[tgt[isp]] * prim
    # neighbour legs
    h = np.einsum("mkl,ilm->ikm", np.conj(C), np.conj(a)) + np.einsum("mlk,ilm->ikm", C, np.conj(a))
    hh = np.ascontiguousarray(np.stack([h.real, h.imag], axis=-1))
    ce = chord_edges(edges_deg)
    K = len(ce) - 1
    gl = np.zeros(len(tgt))
    rc = _lib().orc_neighbor_legs(n, xyz.ctypes.data, delta.ctypes.data, w.ctypes.data, len(piv),
                                  piv.ctypes.data, hh.ctypes.data, K, ce.ctypes.data, int(m_max),
                                  len(tgt), tgt.ctypes.data, gl.ctypes.data)
    if rc != 0:
        raise RuntimeError("orc_neighbor_legs failed (%d)" % rc)
    grad += gl
    if self_pairs == "subtract":
        # d/d(delta_p) of -sum_i w_i d_i sum_k cdiag_k sum_j (w_j d_j)^2 Theta_k(ij):
        # -2 w_p^2 d_p sum_{i in P, p in nbr(i)} w_i d_i cdiag_{k(ip)}, i.e. the neighbour
        # legs with h_m^k = -2 w_p d_p cdiag_k on m = 0 only (divided by w_p, which the
        # legs multiply back in).
        cdiag = np.conj(C)[:, np.arange(K), np.arange(K)].real.sum(axis=0)
        h2 = np.zeros((len(piv), K, int(m_max) + 1, 2))
        h2[:, :, 0, 0] = cdiag[None, :]
        g2 = np.zeros(len(tgt))
        rc = _lib().orc_neighbor_legs(n, xyz.ctypes.data, delta.ctypes.data, w.ctypes.data, len(piv),
                                      piv.ctypes.data, np.ascontiguousarray(h2).ctypes.data, K,
                                      ce.ctypes.data, int(m_max), len(tgt), tgt.ctypes.data,
                                      g2.ctypes.data)
        if rc != 0:
            raise RuntimeError("orc_neighbor_legs failed (%d)" % rc)
        grad -= 2.0 * w[tgt] * delta[tgt] * g2
    return grad


def loss(zeta_c, cot) -> float:
    """L = sum_{m,k1,k2} c Re zeta (the masked-map workload's scalar loss)."""
    return float(np.sum(np.asarray(cot) * np.real(zeta_c)))


def pair_counts(xyz, edges_deg, pivots=None) -> np.ndarray:
    xyz = _f64(xyz)
    n = xyz.shape[0]
    piv = np.arange(n, dtype=np.int64) if pivots is None else _i64a(pivots)
    ce = chord_edges(edges_deg)
    out = np.zeros(len(piv), dtype=np.int64)
    rc = _lib().orc_pair_counts(n, xyz.ctypes.data, len(piv), piv.ctypes.data, len(ce) - 1,
                                ce.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise RuntimeError("orc_pair_counts failed")
    return out


# --------------------------------------------------------------- multi-field

def zeta_multi(xyz, fields, edges_deg, m_max: int, pivots=None):
    """Estimator of three scalar fields A, B, C sampled at the same points (end of
    section 2, after eq. ubEstimator): a pivot field is chosen and the result summed
    over the cyclic permutations of {A, B, C}.  With pivot field P and neighbour fields
    X (first separation bin k1) and Y (second bin k2), the pre-cyclic sums are
        S^{P;XY}_m(k1,k2) = sum_i w^P_i P_i a_m^{k1}(i; X) conj(a_m^{k2}(i; Y)),
        D^{P;XY}(k1,k2)   = sum_i w^P_i W^{k1}(i; X) W^{k2}(i; Y),
    with a(i; X) = sum_j w^X_j X_j e^{-i m phi_ij} and W(i; X) = sum_j w^X_j over the
    bin (the moments of eq. Xm.binned for field X).  Then
        S^{ABC} = S^{A;BC} + S^{B;CA} + S^{C;AB},  D^{ABC} likewise (the same sum with
        every field set to 1, m = 0),  zeta^{ABC} = S^{ABC} / D^{ABC}  (the normalisation contract(norm="R3") applies).
    ``fields`` = ((d_A, w_A), (d_B, w_B), (d_C, w_C)).  S, D and zeta are full K x K
    arrays (not Hermitian unless B = C)."""
    moms = [moments(xyz, d, w, edges_deg, m_max, pivots) for d, w in fields]
    piv = moms[0]["pivots"]
    S = 0.0
    D = 0.0
    for P, X, Y in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        dP, wP = _f64(fields[P][0]), _f64(fields[P][1])
        S = S + np.einsum("i,ikm,ilm->mkl", wP[piv] * dP[piv], moms[X]["a"], np.conj(moms[Y]["a"]))
        D = D + np.einsum("i,ik,il->kl", wP[piv], moms[X]["W"], moms[Y]["W"])
    with np.errstate(divide="ignore", invalid="ignore"):
        zeta = np.where(D[None] != 0, S / np.where(D == 0, 1.0, D)[None], 0.0)
    return dict(S=S, D=D, zeta=zeta, pairs=moms[0]["pairs"], min_margin=moms[0]["min_margin"])


# ------------------------------------------------------------- catalogue D-R

def catalog_zeta(xyz_d, w_d, xyz_r, edges_deg, m_max: int, pivots_d=None, pivots_r=None):
    """Edge-corrected catalogue estimator (the paper is silent; the reading used is the
    Szapudi-Szalay-type D-R ratio).  Data carry x = 1 and weights w_d; randoms carry
    x = -alpha with unit weights, alpha = sum w_d / n_r.  S_m is the estimator over the
    union (pivots and neighbours both); D_R is the d = 1 run over randoms only; then
    zeta = S / (alpha^3 D_R).  ``pivots_d``/``pivots_r`` restrict the pivots (indices into
    each set) for sampled checks.
    """
    nd, nr = len(xyz_d), len(xyz_r)
    alpha = float(np.sum(w_d)) / float(nr)
    xyz = np.concatenate([_f64(xyz_d), _f64(xyz_r)])
    delta = np.concatenate([np.ones(nd), np.full(nr, -alpha)])
    w = np.concatenate([_f64(w_d), np.ones(nr)])
    pd = np.arange(nd) if pivots_d is None else _i64a(pivots_d)
    pr = np.arange(nr) if pivots_r is None else _i64a(pivots_r)
    piv = np.concatenate([pd, nd + pr])
    u = zeta(xyz, delta, w, edges_deg, m_max, piv)
    r = zeta(_f64(xyz_r), np.ones(nr), np.ones(nr), edges_deg, m_max, pr)
    DR = (alpha ** 3) * r["D"]
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(DR[None] != 0, u["S"] / np.where(DR == 0, 1.0, DR)[None], 0.0)
    return dict(S=u["S"], D=DR, zeta=z, alpha=alpha, pairs=u["pairs"] + r["pairs"])


# ------------------------------------------------------------------ m-coupling

def _hermitian_ext(X, n: int):
    """X_n for any integer n from X_0..X_N, with X_{-n} = conj(X_n) (real field)."""
    return X[n] if n >= 0 else np.conj(X[-n])


def edge_correct(S, R, scale: float = 1.0):
    """m-coupling (edge) correction of a data-minus-randoms estimate (the paper leaves
    masks and survey geometry for later; the reading used here is the standard one for
    harmonic 3PCF estimators).

    For one pair of bins the triplet counts are densities in the angle phi between the
    two neighbours, N(phi) for the (D - R) field and R(phi) for the randoms with d = 1,
    and the estimate of the 3PCF is the ratio zeta(phi) = N(phi) / R(phi).  With
    X_n = integral of X(phi) e^{-i n phi} (the raw sums S_n of the estimator, S_{-n} =
    conj(S_n)) and zeta(phi) = sum_m z_m e^{i m phi}, the product becomes a convolution:
        S_m = sum_{m'} z_{m'} scale R_{m - m'},        m = -M..M,
    truncated to |m'| <= M (it needs R_n for n = 0..2M).  ``S`` (M+1, K, K) complex
    (m = 0..M, the D - R run), ``R`` (>= 2M+1, K, K) complex (the randoms' d = 1 run),
    ``scale`` the randoms' normalisation (alpha^3 in the D - R reading).  Solves the
    (2M+1) system per (k1, k2) with numpy.linalg.solve; returns z (M+1, K, K) for
    m = 0..M, 0 where R_0(k1, k2) = 0.  With R_n = 0 for n != 0 (no coupling) this is
    S_m / (scale R_0).
    """
    S = np.asarray(S, dtype=complex)
    R = np.asarray(R, dtype=complex)
    M = S.shape[0] - 1
    K = S.shape[1]
    if R.shape[0] < 2 * M + 1:
        raise ValueError("R needs multipoles 0..2M")
    ms = np.arange(-M, M + 1)
    z = np.zeros((M + 1, K, K), dtype=complex)
    for k1 in range(K):
        for k2 in range(K):
            r = R[:, k1, k2]
            if r[0] == 0:
                continue
            A = np.array([[scale * _hermitian_ext(r, m - mp) for mp in ms] for m in ms])
            b = np.array([_hermitian_ext(S[:, k1, k2], m) for m in ms])
            z[:, k1, k2] = np.linalg.solve(A, b)[M:]
    return z


def catalog_zeta_coupled(xyz_d, w_d, xyz_r, edges_deg, m_max: int, pivots_d=None, pivots_r=None):
    """The D - R catalogue estimate with the m-coupling correction: S from the union
    (as catalog_zeta) at multipoles 0..m_max, R from the randoms' d = 1 run at 0..2 m_max,
    then edge_correct(S, R, alpha^3)."""
    nd, nr = len(xyz_d), len(xyz_r)
    alpha = float(np.sum(w_d)) / float(nr)
    u = catalog_zeta(xyz_d, w_d, xyz_r, edges_deg, m_max, pivots_d, pivots_r)
    pr = np.arange(nr) if pivots_r is None else _i64a(pivots_r)
    r = zeta(_f64(xyz_r), np.ones(nr), np.ones(nr), edges_deg, 2 * m_max, pr)
    z = edge_correct(u["S"], r["S"], alpha ** 3)
    return dict(S=u["S"], R=r["S"], zeta=z, alpha=alpha, zeta_uncorrected=u["zeta"])


# ------------------------------------------------------------------ shared neighbour lists

def ring_pixels(nside: int):
    """(first pixel, pixel count) of each iso-latitude ring of the HEALPix RING scheme,
    north to south (4 nside - 1 rings; Gorski et al. 2005)."""
    out = []
    first = 0
    for r in range(1, 4 * nside):
        n = 4 * r if r < nside else (4 * nside if r <= 3 * nside else 4 * (4 * nside - r))
        out.append((first, n))
        first += n
    return out


def pivot_groups(nside: int, group: int):
    """Each ring's pixels cut into consecutive runs of `group` (the last run of a ring
    shorter); returns (representatives, member lists), the representative of a run being
    its middle pixel, first + (length - 1) // 2."""
    reps, members = [], []
    for first, n in ring_pixels(nside):
        for s in range(0, n, group):
            ln = min(group, n - s)
            reps.append(first + s + (ln - 1) // 2)
            members.append(np.arange(first + s, first + s + ln))
    return np.asarray(reps, dtype=np.int64), members


def zeta_grouped(nside: int, delta, w, edges_deg, m_max: int, group: int, pivots=None):
    """The estimator with shared neighbour lists (Sec. 3.2: pivots very close to one
    another share one neighbour list).  Reading used: the pixels of a ring are cut into
    runs of `group` consecutive pixels (pivot_groups) and every pivot i of a run takes
    the moments of the run's representative rho(i), neighbours and angles both:
        S_m(k1,k2) = sum_i w_i d_i a_m^{k1}(rho(i)) conj(a_m^{k2}(rho(i))),
        D(k1,k2)   = sum_i w_i W^{k1}(rho(i)) W^{k2}(rho(i)),   zeta = S / D,
    over the pivots i in ``pivots`` (default all).  group = 1 is the exact estimator.
    The moments of each representative are those of eq. Xm.binned (all other pixels in
    the bins, the group's own members included)."""
    xyz = pix2vec_ring(nside)
    delta, w = _f64(delta), _f64(w)
    npix = 12 * nside * nside
    use = np.zeros(npix, dtype=bool)
    use[np.arange(npix) if pivots is None else _i64a(pivots)] = True
    reps, members = pivot_groups(nside, group)
    wd = np.array([np.sum((w * delta)[m[use[m]]]) for m in members])
    wt = np.array([np.sum(w[m[use[m]]]) for m in members])
    live = np.array([bool(np.any(use[m])) for m in members])
    reps, wd, wt = reps[live], wd[live], wt[live]
    mom = moments(xyz, delta, w, edges_deg, m_max, reps)
    a, W = mom["a"], mom["W"]
    S = np.einsum("i,ikm,ilm->mkl", wd, a, np.conj(a))
    D = np.einsum("i,ik,il->kl", wt, W, W)
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(D[None] != 0, S / np.where(D == 0, 1.0, D)[None], 0.0)
    return dict(S=S, D=D, zeta=z, reps=reps, min_margin=mom["min_margin"])
