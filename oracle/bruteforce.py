"""Brute-force full-momentum fRG on a small torus -- TEST INFRASTRUCTURE ONLY.

An implementation independent of ``tufrg_oracle.c`` (numpy only, no shared
code) of the *unprojected* one-loop RGE of Sec. 3.1 (Eqs. rg_eq, eq_phipp,
eq_phiphd, eq_phiphc) for the full vertex V_{s1s2s3s4}(k1,k2,k3) on an L x L
mesh, written in the orbital basis via Eq. trafo.  With the complete set of
L*L plane-wave form factors the truncated unity of Eq. unity is exact, so the
channel-decomposed TU-fRG must reproduce these results to rounding; the
tests use that to pin the oracle's loops, projections and V.L.V products.

Regulator reading (same as the oracle): temperature flow, Lambda = T,
chi = 1, so the loops of Eq. def_lmp are d/dT of the bubbles F^-/F^+ of
Eqs. disc_2a/disc_2b.

Array layout: V[k1, k2, k3, s1, s2, s3, s4] with k4 = k1 + k2 - k3 and
momenta as flat indices kx * L + ky.
"""
from __future__ import annotations

import numpy as np


class Torus:
    def __init__(self, spec, mu: float):
        if spec.nc != 1:
            raise ValueError("brute force works on the transfer mesh itself (nc = 1)")
        self.spec = spec
        self.L = L = spec.Lq
        self.N = L * L
        self.ns = spec.n_s
        self.mu = mu
        kx, ky = np.divmod(np.arange(self.N), L)
        self.kvec = np.stack([kx, ky], 1)
        # momentum arithmetic on the torus
        self.add = ((kx[:, None] + kx[None, :]) % L) * L + (ky[:, None] + ky[None, :]) % L
        self.sub = ((kx[:, None] - kx[None, :]) % L) * L + (ky[:, None] - ky[None, :]) % L
        # Bloch Hamiltonian and its eigensystem (library eigh)
        H = np.zeros((self.N, self.ns, self.ns), np.complex128)
        for R, t in zip(spec.hop_R, spec.hop_t):
            ph = np.exp(2j * np.pi * (kx * R[0] + ky * R[1]) / L)
            H += ph[:, None, None] * t[None]
        self.E, self.U = np.linalg.eigh(H)
        self.e = self.E - mu
        # plane-wave form factors f_R(k) = exp(-i k.R) for the bond list
        ff = np.asarray(spec.ff_R)
        self.ff = ff
        self.f = np.exp(-2j * np.pi * (np.outer(kx, ff[:, 0]) + np.outer(ky, ff[:, 1])) / L)  # [k][R]

    # --- Fermi function and the temperature derivatives of the bubbles ---------------------
    @staticmethod
    def _g(e, T):
        x = e / T
        z = np.exp(-np.abs(x))
        h = z / (1 + z) ** 2
        g = x / T * h
        gp = h / T ** 2 * (1 - np.abs(x) * (1 - z) / (1 + z))
        return g, gp

    def w_minus(self, e1, e2, T):
        """d/dT (1 - f(e1) - f(e2)) / (e1 + e2)."""
        g1, gp1 = self._g(e1, T)
        g2, gp2 = self._g(e2, T)
        s = e1 + e2
        deg = np.abs(s) <= 1e-5 * T
        return np.where(deg, -0.5 * (gp1 + gp2), -(g1 + g2) / np.where(deg, 1.0, s))

    def w_plus(self, e1, e2, T):
        """d/dT (f(e1) - f(e2)) / (e1 - e2)."""
        g1, gp1 = self._g(e1, T)
        g2, gp2 = self._g(e2, T)
        d = e1 - e2
        deg = np.abs(d) <= 1e-5 * T
        return np.where(deg, 0.5 * (gp1 + gp2), (g1 - g2) / np.where(deg, 1.0, d))

    def orbital_loops(self, T):
        """L^-_{t1t2t3t4}(k1,k2) and L^+_{t1t2t3t4}(k1,k2), full momentum dependence.

        L^- = sum_l U_{t1l1}(k1) U*_{t3l1}(k1) w^-_{l1l2}(k1,k2) U_{t2l2}(k2) U*_{t4l2}(k2)
        L^+ = sum_l U_{t1l1}(k1) U*_{t3l1}(k1) w^+_{l1l2}(k1,k2) U*_{t2l2}(k2) U_{t4l2}(k2)
        (band loops of Eq. def_lmp dressed by Eq. trafo.)
        """
        e = self.e
        wm = self.w_minus(e[:, None, :, None], e[None, :, None, :], T)   # [k1,k2,l1,l2]
        wp = self.w_plus(e[:, None, :, None], e[None, :, None, :], T)
        U = self.U
        rho = np.einsum("kal,kbl->klab", U, U.conj())                    # rho^l_{ab}(k) = U_al U*_bl
        # l1 rides on k1, l2 on k2
        Lm = np.einsum("xpac,xypq,yqbd->xyabcd", rho, wm, rho, optimize=True)
        Lp = np.einsum("xpac,xypq,yqdb->xyabcd", rho, wp, rho, optimize=True)
        return Lm, Lp

    # --- vertex reconstruction from the exchange propagators -------------------------------
    def k4(self):
        """k4[k1,k2,k3] = k1 + k2 - k3."""
        return self.sub[self.add[:, :, None], np.arange(self.N)[None, None, :]]

    def vertex_from_channels(self, V0, P, C, which="all"):
        """V = V0 + V^P + V^C + V^D (Eq. decom_V) from P(s), C(u) in the matrix layouts.

        V^P(k1,k2,k3) = sum_{RR'} P^{RR'}(k1+k2) f*_R(k1) f_R'(k4)   (Eq. P_1)
        V^C(k1,k2,k3) = sum_{RR'} C^{RR'}(k1-k3) f*_R(k1) f_R'(k4)   (Eq. C_1)
        V^D_{1234}(k1,k2,k3) = -V^C_{1243}(k1,k2,k4)                 (Eq. antisym_cd)
        """
        N, ns, nff = self.N, self.ns, self.ff.shape[0]
        Pt = P.reshape(N, nff, ns, ns, nff, ns, ns)            # [q][R][s1][s2][R'][s4][s3]
        Pt = Pt.transpose(0, 1, 4, 2, 3, 6, 5)                 # [q][R][R'][s1][s2][s3][s4]
        Ct = C.reshape(N, nff, ns, ns, nff, ns, ns)            # [q][R][s1][s3][R'][s4][s2]
        Ct = Ct.transpose(0, 1, 4, 2, 6, 3, 5)                 # [q][R][R'][s1][s2][s3][s4]
        k4 = self.k4()
        fc = self.f.conj()
        V = np.zeros((N, N, N, ns, ns, ns, ns), np.complex128)
        if which in ("all", "0"):
            V += V0[None, None, None]
        # V^P
        s = self.add                                            # [k1,k2]
        if which in ("all", "P"):
            Ps = Pt[s]                                          # [k1,k2][R][R'][s...]
            tmp = np.einsum("xr,xyrtabcd->xytabcd", fc, Ps, optimize=True)
            V += np.einsum("xytabcd,xyzt->xyzabcd", tmp, self.f[k4], optimize=True)
        if which in ("all", "C", "CD"):
            u = self.sub[:, None, :].repeat(N, 1)               # u[k1,k2,k3] = k1 - k3
            Cu = Ct[u]                                          # [k1,k2,k3][R][R']...
            VC = np.einsum("xr,xyzrtabcd,xyzt->xyzabcd", fc, Cu, self.f[k4], optimize=True)
            if which in ("all", "C"):
                V += VC
            if which in ("all", "CD"):
                # V^D_{1234}(k1,k2,k3) = -V^C_{1243}(k1,k2,k4)
                idx3 = k4
                VD = -VC[np.arange(N)[:, None, None], np.arange(N)[None, :, None], idx3].transpose(0, 1, 2, 3, 4, 6, 5)
                V += VD
        return V

    # --- the three one-loop terms ---------------------------------------------------------
    def phi_pp(self, V, Lm):
        """Phi^pp(p1,p2,p3) = -(1/N) sum_{q,t} V_{s1s2t1t2}(p1,p2,q) L^-_{t1t2t3t4}(q,s-q) V_{t3t4s3s4}(q,s-q,p3)."""
        N = self.N
        s = self.add                                            # [p1,p2]
        smq = self.sub[s[:, :, None], np.arange(N)[None, None, :]]   # [p1,p2,q] = s - q
        Lg = Lm[np.arange(N)[None, None, :], smq]               # [p1,p2,q,t1..t4]
        B = V[np.arange(N)[None, None, :], smq]                 # [p1,p2,q,p3,t3,t4,s3,s4]
        return -np.einsum("abqwxij,abqijkl,abqpklyz->abpwxyz", V, Lg, B, optimize=True) / N

    def phi_phc(self, V, Lp):
        """Phi^{ph,c}(p1,p2,p3) = (2/N) sum_{k,t} V_{s1t2s3t1}(p1,k-u,p3) L^+_{t1t2t3t4}(k,k-u) V_{t3s2t4s4}(k,p2,k-u), u = p1-p3."""
        N = self.N
        ar = np.arange(N)
        u = self.sub                                            # [p1,p3]
        kmu = self.sub[ar[None, None, :], u[:, :, None]]        # [p1,p3,k] = k - u
        A2 = V[ar[:, None, None], kmu, ar[None, :, None]]       # [p1,p3,k][s1,t2,s3,t1]
        Lg = Lp[ar[None, None, :], kmu]                         # [p1,p3,k][t1..t4]
        B2 = V[ar[None, None, :, None], ar[None, None, None, :], kmu[:, :, :, None]]  # [p1,p3,k,p2][t3,s2,t4,s4]
        return 2.0 * np.einsum("ackwjyi,ackijmn,ackbmxnz->abcwxyz", A2, Lg, B2, optimize=True) / N

    def phi_phd(self, Phc):
        """Phi^{ph,d}_{1234}(p1,p2,p3) = -Phi^{ph,c}_{1243}(p1,p2,p1+p2-p3) (Eq. eq_phiphc)."""
        N = self.N
        ar = np.arange(N)
        return -Phc[ar[:, None, None], ar[None, :, None], self.k4()].transpose(0, 1, 2, 3, 4, 6, 5)

    # --- channel projections as double k-sums (Eq. def_P and its C, D analogues) -----------
    def project_P(self, V):
        """P^[V]_{RR'}(s) = (1/N^2) sum_{k,k'} f_R(k) f*_R'(k') V(k, s-k, s-k'), in the P matrix layout."""
        N, ns, nff = self.N, self.ns, self.ff.shape[0]
        ar = np.arange(N)
        smk = self.sub[ar[:, None], ar[None, :]]                # [s,k] = s - k
        G = V[ar[None, :, None], smk[:, :, None], smk[:, None, :]]   # [s,k,k'][...]
        out = np.einsum("kr,lt,sklabcd->srtabcd", self.f, self.f.conj(), G, optimize=True) / N ** 2
        # to layout [s][(R,(s1,s2))][(R',(s4,s3))]
        out = out.transpose(0, 1, 3, 4, 2, 6, 5).reshape(N, nff * ns * ns, nff * ns * ns)
        return out

    def project_C(self, V):
        """C^[V]_{RR'}(u) = (1/N^2) sum_{k,k'} f_R(k) f*_R'(k') V(k, k'-u, k-u), in the C matrix layout."""
        N, ns, nff = self.N, self.ns, self.ff.shape[0]
        ar = np.arange(N)
        kmu = self.sub[ar[:, None], ar[None, :]].T              # [u,k] = k - u
        G = V[ar[None, :, None], kmu[:, None, :], kmu[:, :, None]]   # [u,k,k'] = V(k, k'-u, k-u)
        out = np.einsum("kr,lt,uklabcd->urtabcd", self.f, self.f.conj(), G, optimize=True) / N ** 2
        # layout [u][(R,(s1,s3))][(R',(s4,s2))]
        out = out.transpose(0, 1, 3, 5, 2, 6, 4).reshape(N, nff * ns * ns, nff * ns * ns)
        return out

    # --- the full-momentum flow -----------------------------------------------------------
    def dVdT(self, V, T):
        Lm, Lp = self.orbital_loops(T)
        Phc = self.phi_phc(V, Lp)
        return self.phi_pp(V, Lm) + Phc + self.phi_phd(Phc)

    def channel_rhs(self, V, T):
        """(P^[Phi^pp], C^[Phi^{ph,c}]) -- what the channel-decomposed flow must equal."""
        Lm, Lp = self.orbital_loops(T)
        return self.project_P(self.phi_pp(V, Lm)), self.project_C(self.phi_phc(V, Lp))

    def flow_rk4(self, V0, T0, T1, n):
        """Classic RK4 in x = ln T with n equal steps, f = T dV/dT."""
        V = np.broadcast_to(V0[None, None, None], (self.N,) * 3 + V0.shape).astype(np.complex128).copy()
        x, h = np.log(T0), (np.log(T1) - np.log(T0)) / n
        f = lambda xx, VV: np.exp(xx) * self.dVdT(VV, np.exp(xx))
        for _ in range(n):
            k1 = f(x, V)
            k2 = f(x + h / 2, V + h / 2 * k1)
            k3 = f(x + h / 2, V + h / 2 * k2)
            k4 = f(x + h, V + h * k3)
            V = V + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            x += h
        return V

    # --- consistent random states -----------------------------------------------------------
    def swap(self, W, kind):
        """W with legs exchanged: '2134', '1243' or '2143' (momenta and orbitals together)."""
        N = self.N
        ar = np.arange(N)
        k4 = self.k4()
        if kind == "2134":
            return W.transpose(1, 0, 2, 4, 3, 5, 6)
        if kind == "1243":
            return W[ar[:, None, None], ar[None, :, None], k4].transpose(0, 1, 2, 3, 4, 6, 5)
        if kind == "2143":
            return self.swap(self.swap(W, "2134"), "1243")
        raise ValueError(kind)

    def random_consistent_state(self, rng, scale=0.3):
        """(P, C) whose reconstructed vertex has the exchange antisymmetry the flow preserves."""
        N, ns = self.N, self.ns
        shape = (N, N, N, ns, ns, ns, ns)
        W1 = scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
        VP = 0.25 * (W1 - self.swap(W1, "2134") - self.swap(W1, "1243") + self.swap(W1, "2143"))
        W2 = scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
        VC = 0.5 * (W2 + self.swap(W2, "2143"))
        return self.project_P(VP), self.project_C(VC), VP, VC
