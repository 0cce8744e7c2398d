"""CPU FP64 oracle of the RFDiffusion (RFD) graph-field integrator.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this module.  The library
(paper_2302_00942_gb300) never imports, links or runs anything here, and this
module imports nothing from the library: the two share no code.

What it computes (Sec. 2.4 "RFDiffusion", App. A.4):

  graph field integration   i = exp(lambda W) F            (Eq. base_integ, Eq. diffusion)
  eps-NN graph              W(i,j) = f(n_i - n_j)          (Eq. w)
  random features           f(z) = int exp(2 pi i w^T z) tau(w) dw, importance-sampled with p
  real-part estimator       W_hat = (1/h) sum_k cos(2 pi w_k^T z) tau(w_k)/p(w_k)   (App. A.4)
  low-rank identity         exp(lambda A B^T) = I + A [exp(lambda B^T A) - I](B^T A)^{-1} B^T
  evaluation order          x + A([exp(lambda B^T A) - I]((B^T A)^{-1}(B^T x)))

with the readings of the paper used throughout this project:

  * f is the indicator of the L-infinity cube ||z||_inf <= eps: the product of
    per-coordinate sincs printed for tau in Sec. 2.4 is the Fourier transform of
    that cube (an L1 ball's transform does not factor).  With the 2 pi
    convention of Sec. 2.4, tau(w) = prod_d sin(2 pi eps w_d) / (pi w_d)
    (value 2 eps at w_d = 0).  The L2 ball 1[||z||_2 <= eps], whose transform
    Sec. 2.4 names as a Bessel function, is the second threshold function
    (kernel="ball"): tau(w) = 4 pi eps^3 j_1(2 pi eps |w|) / (2 pi eps |w|),
    j_1 the spherical Bessel function of order one.
  * P is a per-coordinate Gaussian N(0, sigma^2) truncated to [-R, R]
    ("(truncated) Gaussian", Sec. 2.4; App. A.4), default sigma = 1/(2 eps),
    R = 1/eps.
  * m counts REAL columns of A and B: h = m/2 frequencies, each giving a cos
    and a sin column, so that A B^T is the real part of phi(n_i)^T psi(n_j).
  * tau/p may be negative, so sqrt(tau/p) is split as A = Phi diag(s sgn r),
    B = Phi diag(s), s = sqrt(2|r|/m): then A B^T = Phi diag(2r/m) Phi^T = W_hat.
  * (B^T A)^{-1} need not exist (N < m); [exp(lambda M) - I] M^{-1} is the
    entire function lambda * phi1(lambda M), phi1(X) = sum_k X^k/(k+1)!,
    which is what is evaluated (never an inverse).

Random numbers (the frequencies w) follow a counter-free published generator,
SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), written out here from its
definition; the library implements the same definition independently.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.special

MASK64 = (1 << 64) - 1
MAX_TRIES = 1 << 20  # rejection-sampling attempts allowed per coordinate


# ---------------------------------------------------------------------------
# Random numbers: SplitMix64 -> 53-bit uniforms in (0, 1)
# ---------------------------------------------------------------------------
class SplitMix64:
    """SplitMix64: a Weyl sequence (increment 0x9E3779B97F4A7C15) passed
    through the variant-13 64-bit finaliser (shifts 30/27/31)."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = int(seed) & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def next_uniform(self) -> float:
        """(top 53 bits + 1/2) * 2^-53: never 0, never 1."""
        return ((self.next_u64() >> 11) + 0.5) * (1.0 / 9007199254740992.0)


def default_sigma(eps: float) -> float:
    return 1.0 / (2.0 * eps)


def default_radius(eps: float) -> float:
    return 1.0 / eps


# ---------------------------------------------------------------------------
# Step a1: frequencies w_j ~ P and weights r_j = tau(w_j)/p(w_j)   (Sec. 2.4)
# ---------------------------------------------------------------------------
def sample_frequencies(m: int, eps: float, seed: int, sigma: float = 0.0,
                       radius: float = 0.0) -> np.ndarray:
    """h = m/2 frequencies in R^3 from the truncated Gaussian P (Sec. 2.4 "Note").

    Per coordinate, independently, in the order j = 0..h-1, d = 0..2: draw
    u1, u2 from the stream; w = R (2 u1 - 1) is uniform on [-R, R]; accept when
    u2 < exp(-(w/sigma)^2 / 2).  Accepted w are exactly N(0, sigma^2)
    conditioned on |w| <= R.
    """
    if m < 2 or m % 2:
        raise ValueError("m must be even and >= 2")
    sigma = sigma or default_sigma(eps)
    radius = radius or default_radius(eps)
    rng = SplitMix64(seed)
    h = m // 2
    omega = np.empty((h, 3), dtype=np.float64)
    for j in range(h):
        for d in range(3):
            for _ in range(MAX_TRIES):
                u1 = rng.next_uniform()
                u2 = rng.next_uniform()
                w = radius * (2.0 * u1 - 1.0)
                a = w / sigma
                if u2 < math.exp(-0.5 * a * a):
                    omega[j, d] = w
                    break
            else:
                raise RuntimeError("rejection sampler did not accept within MAX_TRIES")
    return omega


def tau(omega: np.ndarray, eps: float, kernel: str = "cube") -> np.ndarray:
    """Fourier transform of the threshold function f (Sec. 2.4), 2 pi convention.

    kernel="cube": f = 1[||z||_inf <= eps], the product of per-coordinate sincs,
    prod_d sin(2 pi eps w_d)/(pi w_d).
    kernel="l1_ball": f = 1[||z||_1 <= eps], the octahedron (see below).
    kernel="ball": f = 1[||z||_2 <= eps] in R^3 (the Bessel case of Sec. 2.4):
    the transform of a radial function is radial, and for the ball it is
    (4/3) pi eps^3 * 3 j_1(x)/x with x = 2 pi eps |w| (j_1 from SciPy; the
    value at w = 0 is the ball's volume).
    """
    w = np.asarray(omega, dtype=np.float64)
    if kernel == "l1_ball":
        # f = 1[||z||_1 <= eps] (the L1 ball of Sec. 2.4, an octahedron): the union of
        # the 8 simplices conv(0, s_1 eps e_1, s_2 eps e_2, s_3 eps e_3); over a simplex
        # conv(0, v_1, v_2, v_3), int exp(u.z) dz = 3! vol * exp[0, u.v_1, u.v_2, u.v_3]
        # (divided difference), here with u = -2 pi i w and vol = eps^3 / 6.  The
        # divided difference of exp at nodes x_0..x_3 is the top-right entry of expm of
        # the bidiagonal matrix with the nodes on the diagonal and ones above it (Opitz).
        flat = w.reshape(-1, 3)
        out = np.zeros(len(flat))
        for i, wi in enumerate(flat):
            total = 0.0
            for s in range(8):
                sg = np.array([1.0 if (s >> d) & 1 else -1.0 for d in range(3)])
                nodes = np.concatenate([[0.0], -2j * np.pi * eps * sg * wi])
                J = np.diag(nodes.astype(complex)) + np.diag(np.ones(3, dtype=complex), 1)
                total += scipy.linalg.expm(J)[0, 3].real
            out[i] = eps ** 3 * total
        return out.reshape(w.shape[:-1])
    if kernel == "ball":
        x = 2.0 * np.pi * eps * np.linalg.norm(w, axis=-1)
        safe = np.where(x == 0.0, 1.0, x)
        ratio = np.where(x == 0.0, 1.0 / 3.0, scipy.special.spherical_jn(1, safe) / safe)
        return 4.0 * np.pi * eps ** 3 * ratio
    safe = np.where(w == 0.0, 1.0, w)
    per = np.where(w == 0.0, 2.0 * eps, np.sin(2.0 * np.pi * eps * w) / (np.pi * safe))
    if kernel == "cube_l1":
        # f = ||z||_1 1[||z||_inf <= eps] = sum_d |z_d| prod_e 1[|z_e| <= eps]: the transform is
        # sum_d T(w_d) prod_{e != d} S(w_e), S the sinc above and T the transform of
        # |z| 1[|z| <= eps], 2 int_0^eps z cos(2 pi w z) dz, integrated by parts:
        # T = 2 [eps sin(k eps) / k + (cos(k eps) - 1) / k^2], k = 2 pi w (eps^2 at w = 0;
        # near 0 the same value from the Taylor series of the integrand, to x^10)
        x = 2.0 * np.pi * eps * w
        xs = np.where(np.abs(x) < 0.1, 1.0, x)
        direct = np.sin(xs) / xs + (np.cos(xs) - 1.0) / (xs * xs)
        x2 = x * x
        series = sum(((-1) ** n) * (2 * n + 1) / math.factorial(2 * n + 2) * x2 ** n for n in range(6))
        T = 2.0 * eps * eps * np.where(np.abs(x) < 0.1, series, direct)
        out = np.zeros(w.shape[:-1])
        for d in range(w.shape[-1]):
            term = T[..., d]
            for e in range(w.shape[-1]):
                if e != d:
                    term = term * per[..., e]
            out = out + term
        return out
    if kernel != "cube":
        raise ValueError(f"unknown kernel {kernel!r}")
    return np.prod(per, axis=-1)


def density(omega: np.ndarray, sigma: float, radius: float) -> np.ndarray:
    """pdf of P: per coordinate exp(-w^2/(2 sigma^2)) / (sigma sqrt(2 pi) erf(R/(sigma sqrt 2)))
    on [-R, R] (zero outside)."""
    w = np.asarray(omega, dtype=np.float64)
    norm = sigma * math.sqrt(2.0 * math.pi) * math.erf(radius / (sigma * math.sqrt(2.0)))
    per = np.exp(-0.5 * (w / sigma) ** 2) / norm
    per = np.where(np.abs(w) <= radius, per, 0.0)
    return np.prod(per, axis=-1)


def weights(omega: np.ndarray, eps: float, sigma: float = 0.0, radius: float = 0.0,
            kernel: str = "cube") -> np.ndarray:
    """r_j = tau(w_j) / p(w_j)  (Sec. 2.4: nu_j^2)."""
    sigma = sigma or default_sigma(eps)
    radius = radius or default_radius(eps)
    return tau(omega, eps, kernel) / density(omega, sigma, radius)


# ---------------------------------------------------------------------------
# Step a2: feature map and low-rank factors A, B   (Sec. 2.4, App. A.4)
# ---------------------------------------------------------------------------
def features(points: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """Phi = [cos(2 pi X w^T) | sin(2 pi X w^T)], N x m (real part, App. A.4)."""
    X = np.asarray(points, dtype=np.float64)
    ang = 2.0 * np.pi * (X @ np.asarray(omega, dtype=np.float64).T)
    return np.concatenate([np.cos(ang), np.sin(ang)], axis=1)


def column_scales(r: np.ndarray, m: int) -> tuple[np.ndarray, np.ndarray]:
    """(Omega_a, Omega_b) diagonals: s sgn(r) and s with s = sqrt(2|r|/m),
    each r_j used for its cos and its sin column."""
    s = np.sqrt(2.0 * np.abs(r) / m)
    sa = s * np.sign(r)
    return np.concatenate([sa, sa]), np.concatenate([s, s])


def factors(points: np.ndarray, omega: np.ndarray, r: np.ndarray):
    """A = Phi Omega_a, B = Phi Omega_b with A B^T = W_hat (Sec. 2.4)."""
    m = 2 * omega.shape[0]
    Phi = features(points, omega)
    oa, ob = column_scales(r, m)
    return Phi * oa[None, :], Phi * ob[None, :]


# ---------------------------------------------------------------------------
# Step a4: G = lambda phi1(lambda M) = [exp(lambda M) - I] M^{-1}
# ---------------------------------------------------------------------------
def phi1(X: np.ndarray) -> np.ndarray:
    """phi1(X) = sum_k X^k/(k+1)!, read off the top-right block of
    exp([[X, I], [0, 0]]) = [[e^X, phi1(X)], [0, I]].  SciPy's expm is the
    Al-Mohy--Higham scaling-and-squaring Pade method."""
    X = np.asarray(X, dtype=np.float64)
    k = X.shape[0]
    aug = np.zeros((2 * k, 2 * k))
    aug[:k, :k] = X
    aug[:k, k:] = np.eye(k)
    return scipy.linalg.expm(aug)[:k, k:]


# ---------------------------------------------------------------------------
# The whole estimator, steps a1..a6, in the paper's order
# ---------------------------------------------------------------------------
def rfd_gfi(points, F, eps, lam, m, seed, sigma=0.0, radius=0.0, *, return_parts=False, kernel="cube"):
    """out = F + A (G (B^T F)),  G = lambda phi1(lambda B^T A)  (Sec. 2.4)."""
    F64 = np.asarray(F, dtype=np.float64)
    omega = sample_frequencies(m, eps, seed, sigma, radius)
    r = weights(omega, eps, sigma, radius, kernel)
    A, B = factors(points, omega, r)
    M = B.T @ A                 # m x m   (pre-processing, Sec. 2.4)
    Y = B.T @ F64               # m x c   (inference)
    G = lam * phi1(lam * M)     # m x m   no inverse formed
    out = F64 + A @ (G @ Y)
    if return_parts:
        return out, dict(omega=omega, r=r, A=A, B=B, M=M, Y=Y, G=G)
    return out


def rfd_gfi_from_plan(points, F, lam, omega, r):
    """Same as rfd_gfi for frequencies/weights already drawn (resident plan)."""
    A, B = factors(points, omega, r)
    G = lam * phi1(lam * (B.T @ A))
    F64 = np.asarray(F, dtype=np.float64)
    return F64 + A @ (G @ (B.T @ F64))


# ---------------------------------------------------------------------------
# Brute-force references (small N only)
# ---------------------------------------------------------------------------
def dense_lowrank_gfi(A: np.ndarray, B: np.ndarray, F: np.ndarray, lam: float) -> np.ndarray:
    """exp(lambda A B^T) F with A B^T formed densely (N x N) and exponentiated by
    its symmetric eigendecomposition (LAPACK), no low-rank identity used."""
    W = A @ B.T
    W = 0.5 * (W + W.T)
    e, V = np.linalg.eigh(W)
    return V @ (np.exp(lam * e)[:, None] * (V.T @ np.asarray(F, dtype=np.float64)))


def exact_adjacency(points: np.ndarray, eps: float, kernel: str = "cube") -> np.ndarray:
    """W(i,j) = f(n_i - n_j) (Eq. w): 1[||z||_inf <= eps] (kernel="cube", diagonal 1),
    1[||z||_2 <= eps] ("ball"), ||z||_1 1[||z||_inf <= eps] ("cube_l1", diagonal 0)."""
    X = np.asarray(points, dtype=np.float64)
    diff = X[:, None, :] - X[None, :, :]
    if kernel == "ball":
        return (np.linalg.norm(diff, axis=2) <= eps).astype(np.float64)
    inside = (np.abs(diff).max(axis=2) <= eps).astype(np.float64)
    return inside * np.abs(diff).sum(axis=2) if kernel == "cube_l1" else inside


def dense_exact_gfi(points, F, eps, lam) -> np.ndarray:
    """exp(lambda W) F on the explicit eps-NN graph (the brute-force GFI of
    Sec. 1: materialise the kernel matrix, then multiply)."""
    W = exact_adjacency(points, eps)
    e, V = np.linalg.eigh(W)
    return V @ (np.exp(lam * e)[:, None] * (V.T @ np.asarray(F, dtype=np.float64)))


def smoothed_kernel(z: np.ndarray, eps: float, radius: float) -> np.ndarray:
    """E[W_hat(z)] = int_{[-R,R]^3} exp(2 pi i w^T z) tau(w) dw (App. A.4's f~)
    in closed form: prod_d (1/pi)[Si(2 pi R (eps + z_d)) + Si(2 pi R (eps - z_d))]."""
    z = np.asarray(z, dtype=np.float64)
    si_p = scipy.special.sici(2.0 * np.pi * radius * (eps + z))[0]
    si_m = scipy.special.sici(2.0 * np.pi * radius * (eps - z))[0]
    return np.prod((si_p + si_m) / np.pi, axis=-1)


def smoothed_adjacency(points: np.ndarray, eps: float, radius: float) -> np.ndarray:
    """W~_R(i,j) = f~_R(n_i - n_j), the expectation of W_hat (dense, small N)."""
    X = np.asarray(points, dtype=np.float64)
    return smoothed_kernel(X[:, None, :] - X[None, :, :], eps, radius)


def rel_frobenius(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref||_F / ||ref||_F, the error measure used for every comparison."""
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(x, dtype=np.float64) - ref) / np.linalg.norm(ref))


# ---------------------------------------------------------------------------
# Wasserstein barycenter with the RFD integrator as the kernel action
# (App. C, Algorithm wass_barycenter; Solomon et al. 2015, Algorithm 2)
# ---------------------------------------------------------------------------
BARY_FLOOR = 1e-30  # kernel outputs below this are lifted to it before division / powers


def wasserstein_barycenter(apply_K, mus, area, alpha, iters):
    """Entropic Wasserstein barycenter of the k distributions mus (N x k) with
    weights alpha (k), area weights `area` (N) and the kernel action apply_K
    (x -> K x for an N x k block), following the steps of the algorithm:

        v^i = w^i = 1
        repeat iters times:
            mu = 1
            w^i = mu^i / K(a * v^i)             (step 1)
            d^i = v^i * K(a * w^i)              (step 2)
            mu  = mu * (d^i)^alpha_i            (step 3)
            v^i = v^i * mu / d^i                (step 4, after all i)
        return mu

    mu is reset at the start of each pass (as in Solomon et al.'s Algorithm 2,
    which the paper says it follows); kernel outputs are lifted to BARY_FLOOR
    before they divide or enter a power (the random-feature kernel need not be
    positive).  All k columns of a step go through one kernel action."""
    mus = np.asarray(mus, dtype=np.float64)
    a = np.asarray(area, dtype=np.float64)[:, None]
    alpha = np.asarray(alpha, dtype=np.float64)
    v = np.ones_like(mus)
    mu = np.ones(mus.shape[0])
    for _ in range(iters):
        w = mus / np.maximum(apply_K(a * v), BARY_FLOOR)
        d = v * np.maximum(apply_K(a * w), BARY_FLOOR)
        mu = np.exp(np.log(d) @ alpha)
        v = v * mu[:, None] / d
    return mu


def rfd_barycenter(points, mus, area, alpha, iters, eps, lam, m, seed, sigma=0.0, radius=0.0, kernel="cube"):
    """wasserstein_barycenter with K = exp(lambda W_hat) applied by the low-rank
    identity (the same estimator as rfd_gfi, one plan for every application)."""
    omega = sample_frequencies(m, eps, seed, sigma, radius)
    r = weights(omega, eps, sigma, radius, kernel)
    A, B = factors(points, omega, r)
    G = lam * phi1(lam * (B.T @ A))
    return wasserstein_barycenter(lambda X: X + A @ (G @ (B.T @ X)), mus, area, alpha, iters)


# ---------------------------------------------------------------------------
# Gromov-Wasserstein tensor product and line search with implicit structure
# matrices (App. C.2, Eq. sq, Algorithms tensor_prod and line_search)
# ---------------------------------------------------------------------------
def hadamard_square_action(apply_C, p):
    """C^{(.)2} p = diag(C D_p C^T) (Eq. sq), with two actions of C: apply C to
    D_p (its columns are p_j e_j), transpose, apply C again, take the diagonal."""
    p = np.asarray(p, dtype=np.float64)
    Y = apply_C(np.diag(p))          # C D_p
    Z = apply_C(np.ascontiguousarray(Y.T))   # C (C D_p)^T = C D_p C^T
    return np.diag(Z).copy()


def gw_tensor_product(apply_C, apply_D, T, p, q):
    """L(C, D, T) for the square loss (f1 = f2 = x^2, h1 = x, h2 = 2x),
    Algorithm tensor_prod: w1 = (C^{(.)2} p) 1^T, w2 = 1 (D^{(.)2} q)^T,
    w3 = (FM_D(FM_C(T)^T))^T = C T D^T; return w1 + w2 - 2 w3."""
    T = np.asarray(T, dtype=np.float64)
    v1 = hadamard_square_action(apply_C, p)
    v2 = hadamard_square_action(apply_D, q)
    w3 = apply_D(np.ascontiguousarray(apply_C(T).T)).T
    return v1[:, None] + v2[None, :] - 2.0 * w3


def gw_line_search(apply_C, apply_D, alpha, G, dG, M, p, q):
    """Algorithm line_search: the optimal step tau of a conditional-gradient
    (F)GW iteration, with c_CD from steps 1-2 of tensor_prod,
    a1 = C dG D, b1 = C G D (D symmetric), a = -2 alpha <a1, dG>,
    b = <(1 - alpha) M + alpha c_CD, dG> - 2 alpha (<a1, G> + <b1, dG>).
    Returns (tau, a, b)."""
    G = np.asarray(G, dtype=np.float64)
    dG = np.asarray(dG, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    v1 = hadamard_square_action(apply_C, p)
    v2 = hadamard_square_action(apply_D, q)
    c_cd = v1[:, None] + v2[None, :]
    a1 = apply_D(np.ascontiguousarray(apply_C(dG).T)).T
    b1 = apply_D(np.ascontiguousarray(apply_C(G).T)).T
    a = -2.0 * alpha * float(np.sum(a1 * dG))
    b = float(np.sum(((1.0 - alpha) * M + alpha * c_cd) * dG)) - 2.0 * alpha * (float(np.sum(a1 * G)) +
                                                                              float(np.sum(b1 * dG)))
    if a > 0:
        tau = min(1.0, max(0.0, -b / (2.0 * a)))
    else:
        tau = 1.0 if a + b < 0 else 0.0
    return tau, a, b


def rfd_kernel_action(points, eps, lam, m, seed, sigma=0.0, radius=0.0, kernel="cube"):
    """x -> exp(lambda W_hat) x for the cloud (the FM of one resident plan)."""
    omega = sample_frequencies(m, eps, seed, sigma, radius)
    r = weights(omega, eps, sigma, radius, kernel)
    A, B = factors(points, omega, r)
    G = lam * phi1(lam * (B.T @ A))
    return lambda X: X + A @ (G @ (B.T @ X))


# ---- kernel eigenvalues (Sec. 3.3 point-cloud classification; App. E) --------

def kernel_eigenvalues(A, B, lam, n, k=None, largest=False):
    """The k smallest (largest=False, ascending) or k largest (descending) of
    the N eigenvalues of exp(lam W_hat), W_hat = A B^T (N x N, rank <= m),
    from the low-rank factors (Sec. 3.3: eigenvalues from the factorisation,
    after Nakatsukasa 2019).

    A B^T and the m x m matrix B^T A share their nonzero eigenvalues (with
    multiplicity), so W_hat's spectrum is eig(B^T A) plus N - m zeros when
    N >= m; when N < m, B^T A carries m - N extra zeros (rank <= N), and the
    m - N eigenvalues of smallest modulus are dropped.  exp(lam W_hat) has the
    eigenvalues exp(lam mu) of the same eigenvectors; each zero gives 1.
    W_hat is symmetric, so every mu is real (eig of B^T A by LAPACK; the
    imaginary parts are rounding)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m = A.shape[1]
    mu = np.linalg.eigvals(B.T @ A)
    assert np.all(np.abs(mu.imag) <= 1e-8 * max(1.0, np.abs(mu).max())), "complex eigenvalues"
    mu = mu.real
    if n < m:
        mu = mu[np.argsort(np.abs(mu), kind="stable")[m - n:]]
    kappa = np.concatenate([np.exp(lam * mu), np.ones(max(n - m, 0))])
    kappa = np.sort(kappa)
    if largest:
        kappa = kappa[::-1]
    return kappa[: (n if k is None else k)].copy()


def rfd_kernel_eigenvalues(points, eps, lam, m, seed, k=None, largest=False, sigma=0.0, radius=0.0,
                           kernel="cube"):
    """kernel_eigenvalues of the cloud's RFD factors (same frequencies as rfd_gfi)."""
    omega = sample_frequencies(m, eps, seed, sigma, radius)
    r = weights(omega, eps, sigma, radius, kernel)
    A, B = factors(points, omega, r)
    return kernel_eigenvalues(A, B, lam, len(points), k, largest)
