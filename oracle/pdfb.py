"""Faceted HyperSARA PDFB iteration (Algorithm 2), reweighting (Algorithm 1),
parameters and metrics, float64.

Readings of the paper used here:
  * indicator iota_C is 0 on C and +inf outside (Eq. 3 states it inverted);
  * U_{c,l,b} = I: Euclidean projection onto the l2 balls, eta_l = 1 / ||Phi_l||_S^2;
  * the data dual uses Phi x_check^{(p)} = 2 Phi x^{(p)} - Phi x^{(p-1)} with
    Phi x^{(-1)} := Phi x^{(0)} (the x_hat and v updates of Algorithm 2);
  * P~_{c,q} = D_q P_{c,q} (Algorithm 2 writes P_c);
  * thresholds alpha_j = zeta^-1 mu_bar_q theta_bar_j paired with the singular
    values in descending order; alpha_i = kappa^-1 mu theta_i per wavelet row;
  * the faceted SARA operators sum exactly to the global ones (Section 2.4.2), so
    the iteration applies Psi^dagger / Psi globally; tests pin the equality.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import gammaln

from . import facets as fc
from . import nufft as nu
from . import dde as dd
from . import prox as px
from . import wavelets as wv


# ------------------------------------------------------------------ parameters
def op_norm_sq(uv: np.ndarray, n1: int, n2: int, x0: np.ndarray, max_iter: int = 100,
               rel_tol: float = 1e-4, U: np.ndarray | None = None, dde_k=None) -> float:
    """||Phi||_S^2 on real images by the power method on Re(Phi^dagger Phi)
    (footnote of Section 2.3.1: relative variation below 1e-4, at most 100 iterations);
    with a preconditioner, ||U^1/2 Phi||_S^2 from Re(Phi^dagger U Phi) (Section 3.2);
    dde_k = (kern, kidx of these visibilities): the DDE-extended Phi (Section 2.1)."""
    x = x0 / np.linalg.norm(x0)
    val = 0.0
    for _ in range(max_iter):
        m = nu.measure(x, uv) if dde_k is None else dd.measure(x, uv, dde_k[0], dde_k[1])
        if U is not None:
            m = U * m
        y = (nu.adjoint(m, uv, n1, n2) if dde_k is None else dd.adjoint(m, uv, dde_k[0], dde_k[1], n1, n2)).real
        new = np.linalg.norm(y)
        x = y / new
        if val > 0 and abs(new - val) / new < rel_tol:
            val = new
            break
        val = new
    return float(val)


def noise_sigma(clean_vis: np.ndarray, isnr_db: float) -> float:
    """sigma_l from the iSNR definition of Section 4.1, read per channel:
    iSNR = 10 log10(||Phi_l x_l||^2 / (M_l sigma_l^2))."""
    M = clean_vis.size
    return float(np.linalg.norm(clean_vis) / math.sqrt(M) * 10.0 ** (-isnr_db / 20.0))


def l2_radii(sigma: float, M_b) -> np.ndarray:
    """eps_{l,b} of Eq. (3): eps_l^2 = sigma_l^2 (M_l + 2 sqrt(M_l)), eps_{l,b}^2 = eps_l^2 M_{l,b} / M_l."""
    M_b = np.asarray(M_b, dtype=np.float64)
    M = M_b.sum()
    e2 = sigma ** 2 * (M + 2.0 * math.sqrt(M))
    return np.sqrt(e2 * M_b / M)


def inverse_density(uv: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """U of one channel (Section 3.2): the inverse of the sampling density near each
    acquired Fourier mode, read as 1 / (number of the channel's visibilities whose
    nearest cell of the 2n1 x 2n2 oversampled grid, round(omega K / 2 pi) mod K, is the
    visibility's own)."""
    uv = np.asarray(uv, dtype=np.float64)
    K1, K2 = 2 * n1, 2 * n2
    r = np.floor(uv[:, 1] * K1 / (2.0 * np.pi) + 0.5).astype(np.int64) % K1
    c = np.floor(uv[:, 0] * K2 / (2.0 * np.pi) + 0.5).astype(np.int64) % K2
    cell = r * K2 + c
    _, inv, counts = np.unique(cell, return_inverse=True, return_counts=True)
    return 1.0 / counts[inv]


def chi_mean_std(k: int):
    """Mean and standard deviation of the chi distribution with k degrees of freedom."""
    m = math.sqrt(2.0) * math.exp(gammaln((k + 1) / 2.0) - gammaln(k / 2.0))
    return m, math.sqrt(max(k - m * m, 0.0))


def fhs_heuristics(sigma: np.ndarray, opnorm_sq: np.ndarray, facet_pixels) -> tuple[float, np.ndarray]:
    """mu_c = upsilon_c = sigma_bar_c [m_chi(L_c) + s_chi(L_c)] and
    mu_bar_{c,q} = upsilon_bar_{c,q} = sigma_bar_c sqrt(N~_q L_c / J_{c,q})
    (Section 2.4.2 FHS heuristics), sigma_bar_{c,l} = sigma_{c,l} / ||Phi_{c,l}||_S."""
    sb = np.asarray(sigma) / np.sqrt(np.asarray(opnorm_sq))
    Lc = sb.size
    sbar = math.sqrt(np.mean(sb ** 2))
    m, s = chi_mean_std(Lc)
    mu = sbar * (m + s)
    mu_bar = np.array([sbar * math.sqrt(Nq * Lc / min(Nq, Lc)) for Nq in facet_pixels])
    return mu, mu_bar


# ------------------------------------------------------------------- problem
@dataclass
class Problem:
    """One spectral sub-cube problem (Eq. 5 restricted to sub-cube c)."""
    n1: int
    n2: int
    L: int
    Qy: int
    Qx: int
    rho: float
    window: str
    uv: np.ndarray          # [sum M][2] float32 values, channel-major, block-contiguous
    M_lb: np.ndarray        # [L][B]
    y: np.ndarray           # [sum M] complex
    eps: np.ndarray         # [L][B]
    eta: np.ndarray         # [L]
    mu: float
    mu_bar: np.ndarray      # [Q]
    tau: float = 0.33
    zeta: float = 1.0
    kappa: float = 1.0
    facets: list = field(default_factory=list)
    U: np.ndarray | None = None     # [sum M] diagonal preconditioner (None: U = I)
    n_sub: int = 20                 # forward-backward sub-iterations of the U-projection
    dde: tuple | None = None        # (kern [n_kern][S_d][S_d], kidx [sum M]): DDE-extended G (Section 2.1)

    def __post_init__(self):
        if not self.facets:
            self.facets = fc.nuclear_facets(self.n1, self.n2, self.Qy, self.Qx, self.rho, self.window)

    def vis_slices(self):
        """[(channel, block, slice)] over the channel-major, block-contiguous visibility vector."""
        out, off = [], 0
        for l in range(self.L):
            for b in range(self.M_lb.shape[1]):
                m = int(self.M_lb[l, b])
                out.append((l, b, slice(off, off + m)))
                off += m
        return out

    def channel_slices(self):
        out, off = [], 0
        for l in range(self.L):
            m = int(self.M_lb[l].sum())
            out.append(slice(off, off + m))
            off += m
        return out


@dataclass
class State:
    X: np.ndarray           # [L][n1][n2]
    Xc: np.ndarray          # X_check
    W: np.ndarray           # [L][I]
    theta: np.ndarray       # [I]
    P: list                 # per facet [L][h][w]
    theta_bar: np.ndarray   # [Q][L]
    v: np.ndarray           # [sum M]
    u_prev: np.ndarray      # Phi x^{(p-1)}

    def copy(self):
        return State(self.X.copy(), self.Xc.copy(), self.W.copy(), self.theta.copy(),
                     [p.copy() for p in self.P], self.theta_bar.copy(), self.v.copy(),
                     self.u_prev.copy())


def initial_state(prob: Problem, X0: np.ndarray | None = None) -> State:
    """X^(0) (zero by default), zero duals, unit weights (weights of X = 0 are 1, Section 3.1)."""
    L, n1, n2 = prob.L, prob.n1, prob.n2
    X = np.zeros((L, n1, n2)) if X0 is None else np.array(X0, dtype=np.float64)
    I = wv.n_coefficients(n1, n2)
    P = [np.zeros((L, f["rows"][1] - f["rows"][0], f["cols"][1] - f["cols"][0])) for f in prob.facets]
    u0 = measure_all(prob, X)
    return State(X=X, Xc=X.copy(), W=np.zeros((L, I)), theta=np.ones(I), P=P,
                 theta_bar=np.ones((len(prob.facets), L)), v=np.zeros_like(prob.y), u_prev=u0)


def measure_l(prob: Problem, x: np.ndarray, sl: slice) -> np.ndarray:
    """Phi_l x for the visibilities sl of one channel (DDE-extended G when prob.dde is set)."""
    if prob.dde is None:
        return nu.measure(x, prob.uv[sl])
    return dd.measure(x, prob.uv[sl], prob.dde[0], prob.dde[1][sl])


def adjoint_l(prob: Problem, v: np.ndarray, sl: slice) -> np.ndarray:
    """Phi_l^dagger v (complex image) for the visibilities sl of one channel."""
    if prob.dde is None:
        return nu.adjoint(v, prob.uv[sl], prob.n1, prob.n2)
    return dd.adjoint(v, prob.uv[sl], prob.dde[0], prob.dde[1][sl], prob.n1, prob.n2)


def measure_all(prob: Problem, X: np.ndarray) -> np.ndarray:
    out = np.zeros(prob.uv.shape[0], dtype=np.complex128)
    for l, sl in enumerate(prob.channel_slices()):
        out[sl] = measure_l(prob, X[l], sl)
    return out


# ------------------------------------------------------ Algorithm 2 pieces
def nuclear_step(prob: Problem, Xc: np.ndarray, P: list, theta_bar: np.ndarray):
    """Nuclear duals of all facets and their primal contribution sum_q zeta S~_q^T D_q P_q."""
    L = prob.L
    A = np.zeros_like(Xc)
    newP = []
    for q, f in enumerate(prob.facets):
        (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
        DX = (Xc[:, r0:r1, c0:c1] * D).reshape(L, -1).T
        Pq = P[q].reshape(L, -1).T
        alpha = prob.mu_bar[q] / prob.zeta * theta_bar[q]
        Pn = px.dual_nuclear(Pq, DX, alpha).T.reshape(P[q].shape)
        newP.append(Pn)
        A[:, r0:r1, c0:c1] += prob.zeta * D * Pn
    return newP, A


def sara_step(prob: Problem, Xc: np.ndarray, W: np.ndarray, theta: np.ndarray):
    """l2,1 duals (all facets at once, exact by Section 2.4.2) and kappa Psi W."""
    PsiX = wv.sara_analysis(Xc)                     # [L][I]
    alpha = prob.mu / prob.kappa * theta
    Wn = px.dual_l21(W.T, PsiX.T, alpha).T
    return Wn, prob.kappa * wv.sara_synthesis(Wn, prob.n1, prob.n2)


def data_step(prob: Problem, X: np.ndarray, v: np.ndarray, u_prev: np.ndarray):
    """Data duals of every (channel, block), residual norms and sum_l eta_l Re Phi_l^dagger v_l."""
    u = measure_all(prob, X)
    vn = np.zeros_like(v)
    res = np.zeros(prob.M_lb.shape)
    for (l, b, sl) in prob.vis_slices():
        phixc = 2.0 * u[sl] - u_prev[sl]
        if prob.U is None:
            vn[sl] = px.dual_l2ball(v[sl], phixc, prob.y[sl], prob.eps[l, b])
        else:
            vn[sl] = px.dual_l2ball_precond(v[sl], phixc, prob.y[sl], prob.eps[l, b], prob.U[sl], prob.n_sub)
        res[l, b] = np.linalg.norm(prob.y[sl] - u[sl])
    A = np.zeros_like(X)
    for l, sl in enumerate(prob.channel_slices()):
        A[l] = prob.eta[l] * adjoint_l(prob, vn[sl], sl).real
    return vn, u, res, A


def pdfb_iteration(prob: Problem, st: State) -> dict:
    """One iteration of Algorithm 2 (in place on st); returns xi and the residual norms."""
    P, An = nuclear_step(prob, st.Xc, st.P, st.theta_bar)
    W, As = sara_step(prob, st.Xc, st.W, st.theta)
    v, u, res, Ad = data_step(prob, st.X, st.v, st.u_prev)
    A = An + As + Ad
    Xn = px.proj_nonneg_real(st.X - prob.tau * A)
    xnorm = np.linalg.norm(st.X)
    xi = np.linalg.norm(Xn - st.X) / xnorm if xnorm > 0 else math.inf
    st.Xc = 2.0 * Xn - st.X
    st.X = Xn
    st.P, st.W, st.v, st.u_prev = P, W, v, u
    return {"xi": xi, "res": res, "A_s": As, "A_n": An, "A_d": Ad}


# ------------------------------------------------------ Algorithm 1 weights
def reweight(prob: Problem, X: np.ndarray):
    """theta_i = upsilon / (||[Psi^dagger X]_i||_2 + upsilon) and
    theta_bar_{q,j} = upsilon_bar_q / (s_j(D_q S~_q X) + upsilon_bar_q) (Eqs. 9-10)."""
    PsiX = wv.sara_analysis(X)
    rn = np.linalg.norm(PsiX, axis=0)
    theta = prob.mu / (rn + prob.mu)
    tb = np.zeros((len(prob.facets), prob.L))
    for q, f in enumerate(prob.facets):
        (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
        Z = (X[:, r0:r1, c0:c1] * D).reshape(prob.L, -1).T
        _, s, _ = px.jacobi_svd(Z)
        tb[q] = prob.mu_bar[q] / (s + prob.mu_bar[q])
    return theta, tb


# -------------------------------------------------------------------- metrics
def snr_db(x_true: np.ndarray, x: np.ndarray) -> np.ndarray:
    """SNR_l = 20 log10(||x_true_l|| / ||x_true_l - x_l||) per channel (Section 4.2)."""
    t = x_true.reshape(x_true.shape[0], -1)
    e = (x_true - x).reshape(x_true.shape[0], -1)
    return 20.0 * np.log10(np.linalg.norm(t, axis=1) / np.linalg.norm(e, axis=1))


def snr_log_db(x_true: np.ndarray, x: np.ndarray, eps_img: np.ndarray) -> np.ndarray:
    """SNR_log,l of Section 4.2 with the per-channel image-domain noise level eps_img_l."""
    out = []
    for l in range(x_true.shape[0]):
        a = np.log10(x_true[l] / eps_img[l] + 1.0)
        b = np.log10(np.maximum(x[l], 0.0) / eps_img[l] + 1.0)
        out.append(20.0 * math.log10(np.linalg.norm(a) / np.linalg.norm(a - b)))
    return np.array(out)


# ------------------------------------------------------------ problem set-up
def build_problem(inp, isnr_db: float | None = None, power_iters: int = 100, seed: int = 7) -> tuple[Problem, dict]:
    """Problem of one sub-cube from fhs_synth inputs: noisy data y = Phi x_true + sigma n,
    eps (Eq. 3), eta = 1/||Phi_l||^2, mu, mu_bar (FHS heuristics)."""
    spec = inp.spec
    n = spec.n
    L = inp.x_true.shape[0]
    M_lb = inp.M_lb
    isnr = spec.isnr_db if isnr_db is None else isnr_db
    rng = np.random.default_rng(seed)
    y = np.zeros(inp.uv.shape[0], dtype=np.complex128)
    sig = np.zeros(L)
    opn = np.zeros(L)
    eps = np.zeros(M_lb.shape)
    off = 0
    for l in range(L):
        m = int(M_lb[l].sum())
        sl = slice(off, off + m)
        clean = nu.measure(inp.x_true[l], inp.uv[sl])
        sig[l] = noise_sigma(clean, isnr)
        y[sl] = clean + sig[l] * inp.noise[sl]
        eps[l] = l2_radii(sig[l], M_lb[l])
        opn[l] = op_norm_sq(inp.uv[sl], n, n, rng.standard_normal((n, n)), max_iter=power_iters)
        off += m
    facets = fc.nuclear_facets(n, n, spec.Q, spec.Q, spec.overlap, spec.window)
    npix = [(f["rows"][1] - f["rows"][0]) * (f["cols"][1] - f["cols"][0]) for f in facets]
    mu, mu_bar = fhs_heuristics(sig, opn, npix)
    prob = Problem(n1=n, n2=n, L=L, Qy=spec.Q, Qx=spec.Q, rho=spec.overlap, window=spec.window,
                   uv=inp.uv, M_lb=M_lb, y=y, eps=eps, eta=1.0 / opn, mu=mu, mu_bar=mu_bar,
                   facets=facets)
    return prob, {"sigma": sig, "opnorm_sq": opn}


# --------------------------------------------- Algorithms 1-2 with stopping rules
def solve(prob: Problem, st: State, p_min: int, p_max: int, xi_pdfb: float, res_factor: float,
          t_max: int, xi_reweight: float) -> list:
    """Algorithm 1 around Algorithm 2, in place on st; returns one record per reweighting
    cycle.  Cycle t: weights from X^(t) (Eqs. 9-10); Algorithm 2 restarted from X^(t)
    (X_check^(0) = X^(0), Phi x^(-1) := Phi x^(0)), iterating while p < p_min, or
    p < p_max and (xi > xi_pdfb or ||r|| > res_factor ||eps||), with xi and ||r|| those of
    the last iteration; then xi_rw = ||X^(t+1) - X^(t)||_F / ||X^(t)||_F.  Cycles run while
    t < t_max and xi_rw > xi_reweight (xi_rw = +inf before the first cycle and when
    X^(t) = 0)."""
    eps_norm = float(np.linalg.norm(prob.eps))
    cycles = []
    xi_rw = math.inf
    t = 0
    while t < t_max and xi_rw > xi_reweight:
        st.theta, st.theta_bar = reweight(prob, st.X)
        X_t = st.X.copy()
        st.Xc = st.X.copy()
        st.u_prev = measure_all(prob, st.X)
        p, xi, res = 0, math.inf, math.inf
        while p < p_min or (p < p_max and (xi > xi_pdfb or res > res_factor * eps_norm)):
            out = pdfb_iteration(prob, st)
            xi, res = out["xi"], float(np.linalg.norm(out["res"]))
            p += 1
        nt = np.linalg.norm(X_t)
        xi_rw = float(np.linalg.norm(st.X - X_t) / nt) if nt > 0 else math.inf
        cycles.append({"iterations": p, "xi": xi, "res_norm": res, "xi_rw": xi_rw})
        t += 1
    return cycles


def precondition(prob: Problem, n_sub: int = 20, power_iters: int = 100, seed: int = 7) -> Problem:
    """The preconditioned variant of Section 3.2 on prob (in place): U_{l,b} = inverse
    sampling density of every channel, n_sub forward-backward sub-iterations for the
    U-metric projections, and eta_l = 1 / ||U_l^1/2 Phi_l||_S^2."""
    rng = np.random.default_rng(seed)
    U = np.zeros(prob.uv.shape[0])
    eta = np.zeros(prob.L)
    for l, sl in enumerate(prob.channel_slices()):
        U[sl] = inverse_density(prob.uv[sl], prob.n1, prob.n2)
        eta[l] = 1.0 / op_norm_sq(prob.uv[sl], prob.n1, prob.n2, rng.standard_normal((prob.n1, prob.n2)),
                                  max_iter=power_iters, U=U[sl])
    prob.U, prob.n_sub, prob.eta = U, n_sub, eta
    return prob


def with_dde(prob: Problem, inp, dde_in, sigma: np.ndarray, power_iters: int = 100, seed: int = 9) -> Problem:
    """The DDE-extended measurement model of Section 2.1 on prob (in place): G_l rows are
    the Kaiser-Bessel kernel convolved with each visibility's DDE kernel; the data become
    y = Phi_l x_true + sigma_l n with the same unit noise, and eta_l = 1 / ||Phi_l||_S^2
    of the extended operator."""
    rng = np.random.default_rng(seed)
    prob.dde = (np.asarray(dde_in.kern), np.asarray(dde_in.kidx))
    for l, sl in enumerate(prob.channel_slices()):
        prob.y[sl] = measure_l(prob, inp.x_true[l], sl) + sigma[l] * inp.noise[sl]
        prob.eta[l] = 1.0 / op_norm_sq(prob.uv[sl], prob.n1, prob.n2, rng.standard_normal((prob.n1, prob.n2)),
                                       max_iter=power_iters, dde_k=(prob.dde[0], prob.dde[1][sl]))
    return prob
