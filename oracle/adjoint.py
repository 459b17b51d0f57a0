"""FP64 reference of the unrolled, differentiable plain-LRSTV iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring).  A numpy restatement of
one ADMM iteration of Algorithm 1 (Section III-C) with explicit per-iteration
scalars theta = (tau, alpha, lambda, mu), and its hand-derived adjoint: given
the gradient of a loss with respect to the state after the iteration, the
gradient with respect to the state before it and to theta.  The forward pass
is checked against the C oracle, the adjoint against finite differences of the
C oracle and, for the singular value thresholding, against torch's autograd of
a complex SVD.

State dictionaries hold the cubes of Algorithm 1 as (n1, n2, n3) float64
arrays ("Y", "S", "Z", "L", "G1", "G2") and (3, n1, n2, n3) arrays ("F", "E",
"G3", "G4").

Adjoint of the singular value thresholding R = U f(Sigma) V^H, f(s) =
max(s - t, 0) (eq. E_solution): with P = U^H dA V,
  (U^H dR V)_ij = a_ij P_ij + b_ij conj(P_ji)              (i != j)
  (U^H dR V)_ii = f'(s_i) Re P_ii + i f(s_i)/s_i Im P_ii
  a_ij = (s_j f_j - s_i f_i) / (s_j^2 - s_i^2),  b_ij = (s_i f_j - s_j f_i) / (s_j^2 - s_i^2)
(the differential of the SVD), and the map is self-adjoint under
<X, Y> = Re tr(X^H Y), so the backward applies the same coefficients to
H = U^H G V.  Near-equal singular values use the limits a -> (f + s f')/(2s),
b -> (s f' - f)/(2s).  Directions outside the numerical range of A contribute
(I - U U^H) G V diag(f/s) V^H + U diag(f/s) U^H G (I - V V^H).  The threshold
gradient is -sum_{s_i > t} Re H_ii.
"""
from __future__ import annotations

import numpy as np

__all__ = ["forward_iteration", "backward_iteration", "svt", "svt_backward", "tsvt",
           "tsvt_backward", "diff", "diff_adjoint", "zsolve", "soft", "unrolled_forward",
           "unrolled_backward", "unrolled_loss_grad", "initial_state"]


# ------------------------------------------------------------ operators ---
def diff(x, w):
    """w_n D_n x, circular forward differences along modes 1..3."""
    return np.stack([w[n] * (np.roll(x, -1, axis=n) - x) for n in range(3)])


def diff_adjoint(g, w):
    """sum_n w_n D_n^T g_n with D_n^T g(v) = g(v - e_n) - g(v)."""
    return sum(w[n] * (np.roll(g[n], 1, axis=n) - g[n]) for n in range(3))


def _eig(shape, w):
    a, b, c = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    return sum(w[n] ** 2 * 4 * np.sin(np.pi * idx / shape[n]) ** 2
               for n, idx in enumerate((a, b, c)))


def zsolve(T, mu, w):
    """(mu (I + D_w^* D_w))^{-1} T by the 3-D DFT (eq. Z_solution); symmetric."""
    return np.real(np.fft.ifftn(np.fft.fftn(T) / (mu * (1.0 + _eig(T.shape, w)))))


def soft(x, d):
    return np.sign(x) * np.maximum(np.abs(x) - d, 0.0)


# ------------------------------------------------------------------ SVT ---
def svt(A, t):
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    return (U * np.maximum(s - t, 0.0)) @ Vh


def svt_backward(A, t, G, rtol=1e-12):
    """Returns (dL/dA, dL/dt) for R = SVT_t(A) and dL/dR = G (complex, with
    the real inner product Re tr(X^H Y))."""
    m, n = A.shape
    U, s, Vh = np.linalg.svd(A, full_matrices=True)
    V = Vh.conj().T
    k = min(m, n)
    s = s[:k]
    smax = s.max() if k else 0.0
    r = int(np.sum(s > rtol * max(smax, 1e-300)))   # numerical rank
    Ur, Vr, sr = U[:, :r], V[:, :r], s[:r]
    f = np.maximum(sr - t, 0.0)
    fp = (sr > t).astype(float)
    H = Ur.conj().T @ G @ Vr                        # r x r
    si, sj = sr[:, None], sr[None, :]
    fi, fj = f[:, None], f[None, :]
    fpi = fp[:, None]
    den = sj ** 2 - si ** 2
    close = np.abs(den) <= 1e-9 * np.maximum(si, sj) ** 2
    safe = np.where(close, 1.0, den)
    a = np.where(close, (fi + si * fpi) / (2 * si), (sj * fj - si * fi) / safe)
    b = np.where(close, (si * fpi - fi) / (2 * si), (si * fj - sj * fi) / safe)
    M = a * H + b * H.conj().T
    d = np.diag(H)
    np.fill_diagonal(M, fp * d.real + 1j * (f / sr) * d.imag)
    Abar = Ur @ M @ Vr.conj().T
    q = f / sr
    Pu = np.eye(m) - Ur @ Ur.conj().T
    Pv = np.eye(n) - Vr @ Vr.conj().T
    Abar = Abar + Pu @ G @ Vr @ np.diag(q) @ Vr.conj().T + Ur @ np.diag(q) @ Ur.conj().T @ G @ Pv
    tbar = -float(np.sum(fp * d.real))
    return Abar, tbar


def tsvt(B, t):
    """t-SVT of a real cube: SVT of every frontal slice of fft(B, axis=2)."""
    Bh = np.fft.fft(B, axis=2)
    R = np.stack([svt(Bh[:, :, k], t) for k in range(B.shape[2])], axis=2)
    return np.real(np.fft.ifft(R, axis=2))


def tsvt_backward(B, t, Ebar):
    """Adjoint of tsvt through the complex slices.  E = Re ifft(R) with R_k =
    SVT(fft(B)_k): dL/dR_k = fft(Ebar)_k / n3 (the adjoint of Re ifft), then
    each slice's SVT adjoint, then the adjoint of fft of a real cube,
    dL/dB = Re(n3 ifft(Bhat_bar))."""
    n3 = B.shape[2]
    Bh = np.fft.fft(B, axis=2)
    Gh = np.fft.fft(Ebar, axis=2) / n3
    Bbar_h = np.empty_like(Bh)
    tbar = 0.0
    for k in range(n3):
        Bbar_h[:, :, k], tb = svt_backward(Bh[:, :, k], t, Gh[:, :, k])
        tbar += tb
    Bbar = np.real(np.fft.ifft(Bbar_h, axis=2) * n3)
    return Bbar, tbar


# ------------------------------------------------------------ iteration ---
def initial_state(Y):
    Y = np.asarray(Y, np.float64)
    z3 = np.zeros((3,) + Y.shape)
    return {"Y": Y, "L": Y.copy(), "Z": Y.copy(), "S": np.zeros_like(Y), "G1": np.zeros_like(Y),
            "G2": np.zeros_like(Y), "F": z3.copy(), "E": z3.copy(), "G3": z3.copy(),
            "G4": z3.copy()}


def forward_iteration(st, theta, w=(1.0, 1.0, 1.0)):
    """One iteration of Algorithm 1 (plain LRSTV, Gamma4 updated, printed F
    threshold) with theta = (tau, alpha, lambda, mu).  Returns (new state,
    intermediates for the adjoint)."""
    tau, alpha, lam, mu = theta
    Y, S, Z, G1, G2 = st["Y"], st["S"], st["Z"], st["G1"], st["G2"]
    F, E, G3, G4 = st["F"], st["E"], st["G3"], st["G4"]
    L1 = 0.5 * (Y - S + Z + (G1 - G2) / mu)
    T = mu * L1 + G2 + diff_adjoint(mu * F - G3, w)
    Z1 = zsolve(T, mu, w)
    g = diff(Z1, w)
    a = 0.5 * (g + G3 / mu + E + G4 / mu)
    F1 = soft(a, tau / mu)
    B = F1 - G4 / mu
    E1 = np.stack([tsvt(B[n], alpha / mu) for n in range(3)])
    u = Y - L1 + G1 / mu
    S1 = soft(u, lam / mu)
    new = {"Y": Y, "L": L1, "Z": Z1, "S": S1,
           "G1": G1 + mu * (Y - L1 - S1), "G2": G2 + mu * (L1 - Z1),
           "G3": G3 + mu * (g - F1), "G4": G4 + mu * (E1 - F1), "F": F1, "E": E1}
    inter = {"L1": L1, "T": T, "Z1": Z1, "g": g, "a": a, "F1": F1, "B": B, "E1": E1, "u": u,
             "S1": S1}
    return new, inter


def backward_iteration(st, inter, theta, adj, w=(1.0, 1.0, 1.0)):
    """Adjoint of forward_iteration: adj holds dLoss/d(new state) (missing
    keys are zero); returns (dLoss/d(old state), dLoss/dtheta)."""
    tau, alpha, lam, mu = theta
    Y, S, Z, G1, G2 = st["Y"], st["S"], st["Z"], st["G1"], st["G2"]
    F, E, G3, G4 = st["F"], st["E"], st["G3"], st["G4"]
    L1, T, Z1, g, a, F1, B, E1, u, S1 = (inter[k] for k in
                                          ("L1", "T", "Z1", "g", "a", "F1", "B", "E1", "u", "S1"))
    z = lambda k, sh: adj.get(k, np.zeros(sh))
    sh, sh3 = Y.shape, (3,) + Y.shape
    bL, bZ, bS = z("L", sh).copy(), z("Z", sh).copy(), z("S", sh).copy()
    bF, bE = z("F", sh3).copy(), z("E", sh3).copy()
    bG1n, bG2n, bG3n, bG4n = z("G1", sh), z("G2", sh), z("G3", sh3), z("G4", sh3)
    out = {"Y": z("Y", sh).copy(), "L": np.zeros(sh), "S": np.zeros(sh), "Z": np.zeros(sh),
           "G1": np.zeros(sh), "G2": np.zeros(sh), "F": np.zeros(sh3), "E": np.zeros(sh3),
           "G3": np.zeros(sh3), "G4": np.zeros(sh3)}
    dtau = dalpha = dlam = dmu = 0.0
    # multipliers
    out["G1"] += bG1n
    out["Y"] += mu * bG1n
    bL -= mu * bG1n
    bS -= mu * bG1n
    dmu += np.sum(bG1n * (Y - L1 - S1))
    out["G2"] += bG2n
    bL += mu * bG2n
    bZ -= mu * bG2n
    dmu += np.sum(bG2n * (L1 - Z1))
    out["G3"] += bG3n
    bg = mu * bG3n
    bF -= mu * bG3n
    dmu += np.sum(bG3n * (g - F1))
    out["G4"] += bG4n
    bE += mu * bG4n
    bF -= mu * bG4n
    dmu += np.sum(bG4n * (E1 - F1))
    # S = soft(u, lambda/mu)
    mS = (np.abs(u) > lam / mu).astype(float)
    bu = bS * mS
    sgn = np.sign(u) * mS
    dlam += -np.sum(bS * sgn) / mu
    dmu += np.sum(bS * sgn) * lam / mu ** 2
    out["Y"] += bu
    bL -= bu
    out["G1"] += bu / mu
    dmu += -np.sum(bu * G1) / mu ** 2
    # E = tsvt(F1 - G4/mu, alpha/mu)
    tb_sum = 0.0
    for n in range(3):
        bB, tb = tsvt_backward(B[n], alpha / mu, bE[n])
        bF[n] += bB
        out["G4"][n] -= bB / mu
        dmu += np.sum(bB * G4[n]) / mu ** 2
        tb_sum += tb
    dalpha += tb_sum / mu
    dmu += -tb_sum * alpha / mu ** 2
    # F = soft(a, tau/mu)
    mF = (np.abs(a) > tau / mu).astype(float)
    ba = bF * mF
    sgnF = np.sign(a) * mF
    dtau += -np.sum(bF * sgnF) / mu
    dmu += np.sum(bF * sgnF) * tau / mu ** 2
    bg = bg + 0.5 * ba
    out["G3"] += 0.5 * ba / mu
    out["E"] += 0.5 * ba
    out["G4"] += 0.5 * ba / mu
    dmu += -np.sum(ba * (G3 + G4)) / (2 * mu ** 2)
    # g = D_w Z1
    bZ += diff_adjoint(bg, w)
    # Z1 = zsolve(T, mu)
    bT = zsolve(bZ, mu, w)
    dmu += -np.sum(bZ * Z1) / mu
    # T = mu L1 + G2 + D_w^*(mu F - G3)
    bL += mu * bT
    out["G2"] += bT
    bp = diff(bT, w)
    out["F"] += mu * bp
    out["G3"] -= bp
    dmu += np.sum(bT * L1) + np.sum(bp * F)
    # L1 = (Y - S + Z + (G1 - G2)/mu) / 2
    out["Y"] += 0.5 * bL
    out["S"] -= 0.5 * bL
    out["Z"] += 0.5 * bL
    out["G1"] += 0.5 * bL / mu
    out["G2"] -= 0.5 * bL / mu
    dmu += -np.sum(bL * (G1 - G2)) / (2 * mu ** 2)
    return out, np.array([dtau, dalpha, dlam, dmu])


def unrolled_forward(Y, thetas, w=(1.0, 1.0, 1.0)):
    """K = len(thetas) iterations from the initial state; returns (L_K, tape)."""
    st = initial_state(Y)
    tape = []
    for th in thetas:
        new, inter = forward_iteration(st, th, w)
        tape.append((st, inter, th))
        st = new
    return st["L"], tape


def unrolled_backward(tape, dX, w=(1.0, 1.0, 1.0)):
    """Given dLoss/dL_K, returns (dLoss/dthetas (K x 4), dLoss/dY)."""
    adj = {"L": np.asarray(dX, np.float64)}
    grads = np.zeros((len(tape), 4))
    for k in range(len(tape) - 1, -1, -1):
        s0, inter, th = tape[k]
        adj, grads[k] = backward_iteration(s0, inter, th, adj, w)
    # the initial state is L = Z = Y, so Y also feeds through Z and L
    return grads, adj["Y"] + adj["Z"] + adj["L"]


def unrolled_loss_grad(Y, clean, thetas, w=(1.0, 1.0, 1.0)):
    """Loss = mean((L_K - clean)^2) after K = len(thetas) iterations from the
    initial state; returns (loss, dLoss/dthetas (K x 4), dLoss/dY)."""
    X, tape = unrolled_forward(Y, thetas, w)
    diffL = X - clean
    loss = float(np.mean(diffL ** 2))
    grads, dY = unrolled_backward(tape, 2.0 * diffL / diffL.size, w)
    return loss, grads, dY
