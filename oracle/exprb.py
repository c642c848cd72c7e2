"""exprb43 with Krylov approximations of the phi-function products: the
fourth-order exponential Rosenbrock method (with an embedded third-order
solution) that the paper runs beside Radau IIA (Sec. 2.1, Table "solvers";
Sec. 3.1), written as plainly as numpy allows.

TEST INFRASTRUCTURE ONLY: the test-suite and the benchmark's CPU baseline may
use it; the product path does not.  It shares no code with the CUDA path.

What it computes (readings r22-r24 in the design notes where the paper is
silent):
- the scheme of Hochbruck, Ostermann and Schweitzer (2009), with
  g(u) = F(u) - J_n u and D_i = g(U_i) - g(u_n):
      U2 = u_n + h/2 phi1(h/2 J) F(u_n)
      U3 = u_n + h phi1(h J) F(u_n) + h phi1(h J) D2
      u_{n+1} = u_n + h phi1(h J) F(u_n) + h (16 phi3 - 48 phi4)(h J) D2
                + h (-2 phi3 + 12 phi4)(h J) D3
      embedded: the same with 16 phi3 for D2 and -2 phi3 for D3;
  J_n is the analytical Jacobian at u_n, evaluated once per new point (kept
  across rejected attempts);
- each of the three vectors F(u_n), D2, D3 spans its own Krylov space
  (Arnoldi, modified Gram-Schmidt), built in the inner product of the step's
  error weights D = diag(atol + rtol |u_n|): on D^-1 J D from D^-1 v, so
  that phi_k(tau J) v = D beta V_m phi_k(tau H_m) e1 (Sec. 2.1, after Saad).
  In mass fractions and kelvin J is badly scaled (the temperature row is
  ~1e17 s^-1 on CH4), and the Euclidean Hessenberg's norm then asks for
  40 squarings of its exponential; in the weighted product it reflects the
  chemical time scales;
- the dimension m grows until Saad's leading error term of every product the
  scheme takes from that space, h beta (h h_{m+1,m}) c_k |e_m^T phi_{k+1}(h
  H_m) e1| ||v_{m+1}||_w (c_k the product's coefficient, ||.||_w the RMS norm
  in the error weights, 1/sqrt(N) for the unit basis vector), is at most
  kappa (a non-finite estimate is not below it); or until the space is
  exhausted (h_{m+1,m} <= 1e-13 ||J v_m||, "happy breakdown") or m = N;
- phi_1 .. phi_p(A) e1 from the exponential of the augmented matrix
  [[A, e1, 0], [0, 0, I], [0, 0, 0]] (scipy.linalg.expm, a library primitive);
- the standard step-size control of Hairer, Norsett and Wanner (Vol. I,
  Sec. II.4) on the embedded difference: weights atol + rtol max(|u_n|,
  |u_{n+1}|), h_new = h min(facmax, max(0.2, 0.9 err^(-1/4))), facmax 5 and
  1 right after a rejection; a non-finite stage halves h; the first step
  from the starting-step heuristic the Radau oracle uses.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

# (k, coefficient) of the products each Krylov space supplies
PRODUCTS_F = ((1, 1.0),)
PRODUCTS_D2 = ((1, 1.0), (3, 16.0), (4, 48.0))
PRODUCTS_D3 = ((3, 2.0), (4, 12.0))

STATUS_OK, STATUS_MAX_STEPS, STATUS_H_UNDERFLOW, STATUS_NONFINITE = 0, 1, 2, 4


def phi_vectors(A, p):
    """[phi_1(A) e1, .., phi_p(A) e1]: columns m+1 .. m+p (first m rows) of
    exp([[A, e1, 0], [0, 0, I_{p-1}], [0, 0, 0]])."""
    A = np.atleast_2d(np.asarray(A, dtype=np.float64))
    m = A.shape[0]
    s = m + p
    Ah = np.zeros((s, s))
    Ah[:m, :m] = A
    Ah[0, m] = 1.0
    for j in range(p - 1):
        Ah[m + j, m + j + 1] = 1.0
    E = expm(Ah)
    return [E[:m, m + k] for k in range(p)]


def wrms(v, scal):
    v = np.asarray(v, dtype=np.float64)
    return float(np.sqrt(np.mean((v / scal) ** 2)))


def arnoldi(J, v, h, products, scal, kappa):
    """Arnoldi on J from v with the stopping rule above, in the inner product
    the error weights define: the basis is that of D^-1 J D from D^-1 v,
    D = diag(scal).  Returns (beta, V [N, m], H [m, m], m) of the scaled
    space; beta = 0 and m = 0 for v = 0."""
    J = J * scal[None, :] / scal[:, None]
    v = v / scal
    N = v.shape[0]
    beta = float(np.linalg.norm(v))
    if beta == 0.0:
        return 0.0, np.zeros((N, 0)), np.zeros((0, 0)), 0
    V = np.zeros((N, N + 1))
    H = np.zeros((N + 1, N))
    V[:, 0] = v / beta
    kmax = max(k for k, _ in products)
    for j in range(N):
        w = J @ V[:, j]
        nw = float(np.linalg.norm(w))
        for i in range(j + 1):
            H[i, j] = float(V[:, i] @ w)
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = float(np.linalg.norm(w))
        m = j + 1
        if H[j + 1, j] <= 1e-13 * nw or m == N:
            return beta, V[:, :m], H[:m, :m], m
        V[:, j + 1] = w / H[j + 1, j]
        ph = phi_vectors(h * H[:m, :m], kmax + 1)
        vals = [c * abs(ph[k][m - 1]) for k, c in products]  # ph[k] is phi_{k+1}
        lead = float("nan") if any(np.isnan(vals)) else max(vals)  # no estimate: keep growing
        # v_{m+1} has unit 2-norm in the scaled space: its weighted RMS is 1/sqrt(N)
        est = h * beta * (h * H[j + 1, j]) * lead / np.sqrt(N)
        if est <= kappa:
            return beta, V[:, :m], H[:m, :m], m
    raise AssertionError("unreachable")


def _products(beta, V, H, tau, ks, scal):
    """{k: phi_k(tau J) v} for the (scaled) Krylov space (beta, V, H):
    D beta V phi_k(tau H) e1."""
    if beta == 0.0:
        return {k: np.zeros(V.shape[0]) for k in ks}
    ph = phi_vectors(tau * H, max(ks))
    return {k: scal * (beta * (V @ ph[k - 1])) for k in ks}


def step(f, J, u, fu, h, scal, kappa):
    """One exprb43 attempt from (u, F(u)) with J = J_n: (u_new, u_hat,
    Krylov dimensions, right-hand sides used); u_new None if a stage is not
    finite."""
    b1, V1, H1, m1 = arnoldi(J, fu, h, PRODUCTS_F, scal, kappa)
    half = _products(b1, V1, H1, 0.5 * h, (1,), scal)[1]
    full = _products(b1, V1, H1, h, (1,), scal)[1]
    U2 = u + 0.5 * h * half
    F2 = f(U2)
    if not np.all(np.isfinite(F2)):
        return None, None, (m1, 0, 0), 1
    D2 = F2 - fu - J @ (U2 - u)
    b2, V2, H2, m2 = arnoldi(J, D2, h, PRODUCTS_D2, scal, kappa)
    q = _products(b2, V2, H2, h, (1, 3, 4), scal)
    U3 = u + h * full + h * q[1]
    F3 = f(U3)
    if not np.all(np.isfinite(F3)):
        return None, None, (m1, m2, 0), 2
    D3 = F3 - fu - J @ (U3 - u)
    b3, V3, H3, m3 = arnoldi(J, D3, h, PRODUCTS_D3, scal, kappa)
    r = _products(b3, V3, H3, h, (3, 4), scal)
    base = u + h * full
    unew = base + h * (16.0 * q[3] - 48.0 * q[4]) + h * (-2.0 * r[3] + 12.0 * r[4])
    uhat = base + h * (16.0 * q[3]) + h * (-2.0 * r[3])
    return unew, uhat, (m1, m2, m3), 2


def integrate(f, jac, y0, t1, *, rtol=1e-6, atol=1e-10, kappa=0.1, h0=None, hfixed=0.0,
              max_steps=100000):
    """exprb43 from t = 0 to t1.  hfixed > 0: constant steps (clipped onto
    t1), every step accepted (for order tests).  Returns (y, stats)."""
    from oracle import oracle as O
    y = np.array(y0, dtype=np.float64)
    N = y.shape[0]
    st = dict(nstep=0, naccpt=0, nrejct=0, nfcn=0, njac=0, krylov=0, krylov_max=0,
              status=STATUS_OK)
    fy = np.asarray(f(y), dtype=np.float64)
    st["nfcn"] += 1
    if not np.all(np.isfinite(fy)):
        st["status"] = STATUS_NONFINITE
        return y, st
    J = np.asarray(jac(y), dtype=np.float64)
    st["njac"] += 1
    if hfixed > 0.0:
        h = hfixed
    elif h0 is not None:
        h = h0
    else:
        h, nf = O.initial_step(lambda t, v: f(v), y, 0.0, t1, rtol, atol)
        st["nfcn"] += nf
    x, facmax, last = 0.0, 5.0, False
    while True:
        if st["nstep"] >= max_steps:
            st["status"] = STATUS_MAX_STEPS
            return y, st
        if 0.1 * abs(h) <= abs(x) * 1e-16:
            st["status"] = STATUS_H_UNDERFLOW
            return y, st
        if x + 1.0001 * h >= t1:
            h = t1 - x
            last = True
        st["nstep"] += 1
        scal = atol + rtol * np.abs(y)
        unew, uhat, ms, nf = step(f, J, y, fy, h, scal, kappa)
        st["nfcn"] += nf
        st["krylov"] += sum(ms)
        st["krylov_max"] = max(st["krylov_max"], *ms)
        if unew is None:
            st["nrejct"] += 1
            h *= 0.5
            last = False
            facmax = 1.0
            continue
        err = wrms(unew - uhat, atol + rtol * np.maximum(np.abs(y), np.abs(unew)))
        err = max(err, 1e-10)
        fac = 0.9 * err ** -0.25
        if hfixed > 0.0 or err <= 1.0:
            x = t1 if last else x + h
            y = unew
            st["naccpt"] += 1
            if last:
                return y, st
            fy = np.asarray(f(y), dtype=np.float64)
            st["nfcn"] += 1
            if not np.all(np.isfinite(fy)):
                st["status"] = STATUS_NONFINITE
                return y, st
            J = np.asarray(jac(y), dtype=np.float64)
            st["njac"] += 1
            if hfixed <= 0.0:
                h = h * min(facmax, max(0.2, fac))
            facmax = 5.0
        else:
            st["nrejct"] += 1
            h = h * max(0.2, fac)
            facmax = 1.0
            last = False


def integrate_states(mech, states, dt, *, rtol=1e-6, atol=1e-10, kappa=0.1, hfixed=0.0):
    """exprb43 on each reactor state (the mass-fraction form, the oracle's
    orc_rhs / orc_jac).  Returns (Y [ns, n], T [n], stats list)."""
    from oracle import oracle as O
    om = O.OracleMech(mech)
    n = states.n
    Y = np.array(states.Y, dtype=np.float64)
    T = np.array(states.T, dtype=np.float64)
    out = []
    for i in range(n):
        P = float(states.P[i])
        f = lambda v: O.rhs(om, P, v)[0]
        jac = lambda v: O.jac(om, P, v)[0]
        y0 = np.concatenate([[T[i]], Y[:-1, i]])
        y, st = integrate(f, jac, y0, dt, rtol=rtol, atol=atol, kappa=kappa, hfixed=hfixed)
        T[i] = y[0]
        Y[:-1, i] = y[1:]
        Y[-1, i] = 1.0 - y[1:].sum()
        out.append(st)
    return Y, T, out
