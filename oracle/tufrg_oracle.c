/*
 * tufrg_oracle.c -- plain FP64 CPU oracle of the TU-fRG right-hand side and flow.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline and reference legs of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; both read the
 * same model descriptor (bonds, hoppings, V0, meshes) and nothing else.
 *
 * What it computes, step by step, in the paper's order and notation
 * (Schober, Ehrlich, Reckling, Honerkamp, "Truncated-unity functional
 * renormalization group for multiband systems with spin-orbit coupling"):
 *
 *  1. H(k) on the fine mesh from the hopping list and its eigensystem
 *     H(k) U = U diag(E), e_l(k) = E_l(k) - mu (Sec. 3, text after Eq. disc_2b),
 *     by a complex Jacobi eigensolver written here.
 *  2. mu by bisection of the filling at a fixed temperature (the paper is
 *     silent; reading: mu fixed once and held constant).
 *  3. Orbital loops by the direct fine-mesh k-sum (Eqs. loopminus/loopplus
 *     transcribed to the orbital basis with Eq. trafo, cf. Eq. loop_orbital).
 *     Regulator (Eq. def_lmp): temperature flow, Lambda = T, chi = 1,
 *     L = d/dT F (Eqs. disc_2a, disc_2b); or the momentum-shell regulator the
 *     paper writes, chi_Lambda(e) = e^2 / (e^2 + Lambda^2) (a smooth
 *     suppression of |e| < Lambda around the Fermi surfaces), with
 *     L = d/dLambda [chi_Lambda(e1) chi_Lambda(e2)] F(e1, e2) and F at a fixed
 *     temperature.
 *  4. Lattice Fourier transform of P and C (Sec. 3.3, after Eq. zw_1).
 *  5. Projections A_P, A_C from Eq. sum_P and the four printed gathers
 *     (Eq. proj_PD, the D->P formula after it, the P->C formula and
 *     Eq. proj_DC), each evaluated literally.
 *  6. dP/dT = A_P L^- A_P (Eq. RGE_spin), dC/dT = 2 A_C L^+ A_C (orbital
 *     form of Eq. rge_Dmat), by naive triple loops.
 *  7. Dormand-Prince 5(4) integration in ln T (the paper names no integration
 *     scheme; this one is the implementation's choice).
 *  8. Band-basis exchange propagators from the orbital ones with the
 *     transformation matrices U(s), X(u) (Sec. 3.4, Eqs. trafo_P,
 *     mat_trafo_P, mat_trafo_D), from their k-sum definitions.
 *
 * Parity status of each function is pinned by tests under tests/ (see the
 * oracle pin tests); nothing here is unpinned.  A mutation test compiles
 * copies of this file with one planted mistake each (a dropped term, a wrong
 * sign, index, momentum or conjugation, a mistyped coefficient) and requires
 * every copy to fail a pin.
 *
 * Index layouts (all complex numbers stored as interleaved re,im doubles):
 *   E[k][l], U[k][tau][l]                      fine mesh k = kx*Lf + ky
 *   Lc[q][d][a][b]                             compact loop, d indexes the sorted
 *                                              list of bond differences R1-R2,
 *                                              a,b pair indices as in the matrices
 *   X[ch][q][M][M], M = n_ff * ns^2           ch 0 = P, ch 1 = C
 *     P row (R,(s1,s2)) col (R',(s4,s3)) holds P^{RR'}_{s1 s2 s3 s4}
 *     C row (R,(s1,s3)) col (R',(s4,s2)) holds C^{RR'}_{s1 s2 s3 s4}
 *   P-loop matrix  [(R1,(t2,t1)),(R2,(t4,t3))] = [L^-_{t1 t2 t3 t4}]_{R1 R2}
 *   C-loop matrix  [(R1,(t1,t2)),(R2,(t3,t4))] = [L^+_{t1 t2 t3 t4}]_{R1 R2}
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int ns;            /* spin-orbitals */
    int nhop;
    const int *hopR;   /* [nhop][2] */
    const double *hopt;/* [nhop][ns][ns] complex */
    const double *V0;  /* [ns]^4 complex */
    int nff;
    const int *ffR;    /* [nff][2] */
    int Lq, nc;
    double mu;
    int reg;           /* 0: temperature flow (scale = T); 1: momentum shell (scale = Lambda) */
    double T_reg;      /* momentum shell: temperature of the Fermi functions in F */
    const double *V0q; /* NULL, or [2][Nq][M][M] complex: the projected bare vertex P^[V0](q), C^[V0](q) in the
                          layouts of the state, used in place of the onsite V0 (the band-basis flow, where the
                          bare vertex depends on the momenta) */
} or_model;

static const double TWO_PI = 6.283185307179586476925286766559;

static int imod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

/* exp(i * 2 pi * n / L) with the integer reduced first, so equal lattice
 * phases are bit-identical. */
static cplx lattice_phase(long n, int L)
{
    long r = n % L; if (r < 0) r += L;
    double a = TWO_PI * (double)r / (double)L;
    return cos(a) + I * sin(a);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1. Hermitian eigensolver: cyclic complex Jacobi                           */
/* ------------------------------------------------------------------------ */

/* H: n x n Hermitian (row-major, interleaved complex), destroyed.
 * On return E ascending, columns of U the eigenvectors (H U = U diag E). */
static void jacobi_herm(int n, cplx *A, double *E, cplx *V)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    double scale = 0.0;
    for (int i = 0; i < n * n; i++) scale += creal(A[i] * conj(A[i]));
    scale = sqrt(scale);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off += creal(A[p * n + q] * conj(A[p * n + q]));
        if (sqrt(off) <= 1e-15 * (scale > 0 ? scale : 1.0)) break;
        for (int p = 0; p < n; p++) {
            for (int q = p + 1; q < n; q++) {
                cplx apq = A[p * n + q];
                double r = cabs(apq);
                if (r < 1e-300) continue;
                /* step 1: phase so that A_pq becomes real: D = diag(.., 1 (p), e^{-i phi} (q), ..)
                 * A <- D^H A D scales row q by e^{+i phi}, column q by e^{-i phi}. */
                cplx ph = apq / r;          /* e^{i phi} */
                for (int k = 0; k < n; k++) {
                    A[q * n + k] *= ph;       /* row q times e^{i phi} */
                }
                for (int k = 0; k < n; k++) {
                    A[k * n + q] *= conj(ph); /* column q times e^{-i phi} */
                }
                for (int k = 0; k < n; k++) V[k * n + q] *= conj(ph);
                /* step 2: real symmetric rotation on (p,q) */
                double app = creal(A[p * n + p]), aqq = creal(A[q * n + q]);
                double theta = (aqq - app) / (2.0 * r);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J_pp = c, J_pq = s, J_qp = -s, J_qq = c */
                for (int k = 0; k < n; k++) {
                    cplx akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    cplx apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                A[p * n + q] = 0.0; A[q * n + p] = 0.0;
                for (int k = 0; k < n; k++) {
                    cplx vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    /* sort ascending (selection sort, stable for equal values) */
    for (int i = 0; i < n; i++) E[i] = creal(A[i * n + i]);
    for (int i = 0; i < n; i++) {
        int m = i;
        for (int j = i + 1; j < n; j++) if (E[j] < E[m]) m = j;
        if (m != i) {
            double te = E[i]; E[i] = E[m]; E[m] = te;
            for (int k = 0; k < n; k++) { cplx tv = V[k * n + i]; V[k * n + i] = V[k * n + m]; V[k * n + m] = tv; }
        }
    }
}

void or_eigh(int n, const double *H, double *E, double *U)
{
    cplx *A = malloc(sizeof(cplx) * n * n);
    memcpy(A, H, sizeof(cplx) * n * n);
    jacobi_herm(n, A, E, (cplx *)U);
    free(A);
}

/* H(k) = sum_R t_R e^{i k.R}, k = 2 pi (kx, ky) / Lf (Sec. 3.1: Bloch Hamiltonian). */
static void bloch_h(const or_model *m, int Lf, int kx, int ky, cplx *H)
{
    int ns = m->ns;
    const cplx *t = (const cplx *)m->hopt;
    for (int i = 0; i < ns * ns; i++) H[i] = 0.0;
    for (int h = 0; h < m->nhop; h++) {
        cplx ph = lattice_phase((long)kx * m->hopR[2 * h] + (long)ky * m->hopR[2 * h + 1], Lf);
        for (int i = 0; i < ns * ns; i++) H[i] += t[h * ns * ns + i] * ph;
    }
}

/* Eigensystem on the fine mesh.  E [Nk][ns], U [Nk][ns][ns] (row tau, column band). */
void or_bands(const or_model *m, double *E, double *U)
{
    int ns = m->ns, Lf = m->Lq * m->nc, Nk = Lf * Lf;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < Nk; k++) {
        cplx H[64], V[64];
        bloch_h(m, Lf, k / Lf, k % Lf, H);
        jacobi_herm(ns, H, E + (size_t)k * ns, V);
        memcpy(U + (size_t)k * ns * ns * 2, V, sizeof(cplx) * ns * ns);
    }
}

/* ------------------------------------------------------------------------ */
/* 2. Fermi function, its temperature derivatives, mu                         */
/* ------------------------------------------------------------------------ */

/* f(e) = 1/(e^{e/T}+1) (Sec. 3.1).  Written with z = e^{-|e|/T} so it never overflows. */
static double fermi(double e, double T)
{
    double z = exp(-fabs(e) / T);
    return e > 0 ? z / (1.0 + z) : 1.0 / (1.0 + z);
}

/* g = d f / dT = (e/T^2) f (1-f);  gp = d g / d e = (f(1-f)/T^2)(1 - (e/T) tanh(e/2T)). */
static void fermi_dT(double e, double T, double *g, double *gp)
{
    double x = e / T, ax = fabs(x);
    double z = exp(-ax);
    double h = z / ((1.0 + z) * (1.0 + z));          /* f(1-f) */
    *g = x / T * h;
    *gp = h / (T * T) * (1.0 - ax * (1.0 - z) / (1.0 + z));
}

void or_fermi(double e, double T, double *f, double *g, double *gp)
{
    *f = fermi(e, T);
    fermi_dT(e, T, g, gp);
}

/* Degenerate-pair switch: below |delta| = 1e-5 T use the trapezoid of g'. */
#define OR_DEGEN 1e-5

/* d/dT F^-(e1,e2), F^- = (1 - f(e1) - f(e2))/(e1 + e2)  (Eq. disc_2a). */
double or_wm(double e1, double e2, double T)
{
    double g1, g2, gp1, gp2;
    fermi_dT(e1, T, &g1, &gp1);
    fermi_dT(e2, T, &g2, &gp2);
    double s = e1 + e2;
    if (fabs(s) > OR_DEGEN * T) return -(g1 + g2) / s;
    return -0.5 * (gp1 + gp2);
}

/* d/dT F^+(e1,e2), F^+ = (f(e1) - f(e2))/(e1 - e2)  (Eq. disc_2b). */
double or_wp(double e1, double e2, double T)
{
    double g1, g2, gp1, gp2;
    fermi_dT(e1, T, &g1, &gp1);
    fermi_dT(e2, T, &g2, &gp2);
    double d = e1 - e2;
    if (fabs(d) > OR_DEGEN * T) return (g1 - g2) / d;
    return 0.5 * (gp1 + gp2);
}

/* The bubbles themselves (not their T-derivative), for the closed-form pins. */
double or_Fm(double e1, double e2, double T)
{
    double s = e1 + e2;
    if (fabs(s) > OR_DEGEN * T) return (1.0 - fermi(e1, T) - fermi(e2, T)) / s;
    /* limit e2 -> -e1: -(d f / d e)(e1) = f(1-f)/T */
    double f1 = fermi(e1, T), f2 = fermi(-e2, T);
    return 0.5 * (f1 * (1 - f1) + f2 * (1 - f2)) / T;
}

double or_Fp(double e1, double e2, double T)
{
    double d = e1 - e2;
    if (fabs(d) > OR_DEGEN * T) return (fermi(e1, T) - fermi(e2, T)) / d;
    double f1 = fermi(e1, T), f2 = fermi(e2, T);
    return -0.5 * (f1 * (1 - f1) + f2 * (1 - f2)) / T;
}

/* Momentum-shell regulator of Eq. def_lmp: chi_Lambda(e) = e^2 / (e^2 + Lambda^2) and its
 * Lambda-derivative -2 Lambda e^2 / (e^2 + Lambda^2)^2. */
double or_chi(double e, double lam) { return e * e / (e * e + lam * lam); }
double or_dchi(double e, double lam)
{
    double d = e * e + lam * lam;
    return -2.0 * lam * e * e / (d * d);
}

/* L^-/+ weight with the momentum-shell regulator: d/dLambda [chi(e1) chi(e2)] F^-/+(e1, e2) at T. */
double or_wm_shell(double e1, double e2, double lam, double T)
{
    return (or_dchi(e1, lam) * or_chi(e2, lam) + or_chi(e1, lam) * or_dchi(e2, lam)) * or_Fm(e1, e2, T);
}
double or_wp_shell(double e1, double e2, double lam, double T)
{
    return (or_dchi(e1, lam) * or_chi(e2, lam) + or_chi(e1, lam) * or_dchi(e2, lam)) * or_Fp(e1, e2, T);
}

/* The loop weight of channel `which' at scale s (T or Lambda): kind 0 the flowing loop, kind 1 the
 * quantity whose s-derivative it is (the bubble F, or chi chi F with the momentum shell). */
static double loop_weight(const or_model *m, int which, int kind, double a, double b, double s)
{
    if (m->reg == 1) {
        if (kind) return or_chi(a, s) * or_chi(b, s) * (which == 0 ? or_Fm(a, b, m->T_reg) : or_Fp(a, b, m->T_reg));
        return which == 0 ? or_wm_shell(a, b, s, m->T_reg) : or_wp_shell(a, b, s, m->T_reg);
    }
    if (which == 0) return kind ? or_Fm(a, b, s) : or_wm(a, b, s);
    return kind ? or_Fp(a, b, s) : or_wp(a, b, s);
}

/* n(mu) = (1/Nk) sum_{k,l} f(E_l(k) - mu): electrons per site. */
double or_density(const or_model *m, const double *E, double mu, double T)
{
    int ns = m->ns, Lf = m->Lq * m->nc, Nk = Lf * Lf;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int k = 0; k < Nk; k++)
        for (int l = 0; l < ns; l++) s += fermi(E[(size_t)k * ns + l] - mu, T);
    return s / Nk;
}

/* Bisection of n(mu) = filling on [min E - 1, max E + 1], 200 halvings. */
double or_find_mu(const or_model *m, const double *E, double filling, double T)
{
    int ns = m->ns, Lf = m->Lq * m->nc, Nk = Lf * Lf;
    double lo = E[0], hi = E[0];
    for (size_t i = 0; i < (size_t)Nk * ns; i++) { if (E[i] < lo) lo = E[i]; if (E[i] > hi) hi = E[i]; }
    lo -= 1.0; hi += 1.0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (or_density(m, E, mid, T) < filling) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* bond bookkeeping                                                           */
/* ------------------------------------------------------------------------ */

/* Sorted list (by dx, then dy) of the distinct differences R1 - R2 over the bond set. */
int or_delta_list(const or_model *m, int *out)
{
    int n = 0;
    for (int i = 0; i < m->nff; i++)
        for (int j = 0; j < m->nff; j++) {
            int dx = m->ffR[2 * i] - m->ffR[2 * j], dy = m->ffR[2 * i + 1] - m->ffR[2 * j + 1];
            int seen = 0;
            for (int c = 0; c < n; c++) if (out[2 * c] == dx && out[2 * c + 1] == dy) { seen = 1; break; }
            if (!seen) { out[2 * n] = dx; out[2 * n + 1] = dy; n++; }
        }
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++)
            if (out[2 * j] < out[2 * i] || (out[2 * j] == out[2 * i] && out[2 * j + 1] < out[2 * i + 1])) {
                int tx = out[2 * i], ty = out[2 * i + 1];
                out[2 * i] = out[2 * j]; out[2 * i + 1] = out[2 * j + 1];
                out[2 * j] = tx; out[2 * j + 1] = ty;
            }
    return n;
}

static int delta_index(const int *dl, int nd, int dx, int dy)
{
    for (int c = 0; c < nd; c++) if (dl[2 * c] == dx && dl[2 * c + 1] == dy) return c;
    return -1;
}

/* index of the bond congruent to (x, y) modulo Lq, or -1 */
static int ff_index_mod(const or_model *m, int x, int y)
{
    int L = m->Lq;
    for (int i = 0; i < m->nff; i++)
        if (imod(m->ffR[2 * i] - x, L) == 0 && imod(m->ffR[2 * i + 1] - y, L) == 0) return i;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* 3. orbital loops by the direct k-sum                                       */
/* ------------------------------------------------------------------------ */

/*
 * which = 0 (particle-particle, s on the coarse mesh):
 *   [L^-_{t1t2t3t4}(s)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)}
 *        sum_{l1 l2} U_{t1 l1}(s-q) U*_{t3 l1}(s-q) w^-_{l1 l2}(s-q, q) U_{t2 l2}(q) U*_{t4 l2}(q)
 * which = 1 (crossed particle-hole, u on the coarse mesh):
 *   [L^+_{t1t2t3t4}(u)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)}
 *        sum_{l1 l2} U_{t1 l1}(q) U*_{t3 l1}(q) w^+_{l1 l2}(q, q-u) U*_{t2 l2}(q-u) U_{t4 l2}(q-u)
 * kind = 0: w = the flowing loop at scale T (d/dT F, Eq. def_lmp with chi = 1 and Lambda = T), or at
 *           Lambda with the momentum-shell regulator (d/dLambda [chi chi] F, see loop_weight)
 * kind = 1: w = F itself, or chi chi F (the bubbles, used only by the closed-form pins).
 * Output Lc[q][d][a][b] in the matrix pair order given in the file header.
 */
/* the k-sum for one transfer momentum s (coarse index), accumulated into acc[nd][ns^4] */
static void loops_one(const or_model *m, const double *E, const cplx *U, double T, int which, int kind, int s,
                      int nd, const cplx *ph_tab, cplx *acc)
{
    int ns = m->ns, ns2 = ns * ns, ns4 = ns2 * ns2;
    int Lq = m->Lq, nc = m->nc, Lf = Lq * nc, Nk = Lf * Lf;
    int sx = (s / Lq) * nc, sy = (s % Lq) * nc;   /* transfer momentum on the fine mesh */
    cplx *Y = malloc(sizeof(cplx) * ns4);
    double *w = malloc(sizeof(double) * ns2);
    for (size_t i = 0; i < (size_t)nd * ns4; i++) acc[i] = 0.0;
    for (int qx = 0; qx < Lf; qx++)
        for (int qy = 0; qy < Lf; qy++) {
            int k1, k2;
            if (which == 0) { k1 = imod(sx - qx, Lf) * Lf + imod(sy - qy, Lf); k2 = qx * Lf + qy; }
            else            { k1 = qx * Lf + qy; k2 = imod(qx - sx, Lf) * Lf + imod(qy - sy, Lf); }
            const double *e1 = E + (size_t)k1 * ns, *e2 = E + (size_t)k2 * ns;
            const cplx *U1 = U + (size_t)k1 * ns2, *U2 = U + (size_t)k2 * ns2;
            for (int l1 = 0; l1 < ns; l1++)
                for (int l2 = 0; l2 < ns; l2++) {
                    double a = e1[l1] - m->mu, b = e2[l2] - m->mu;
                    w[l1 * ns + l2] = loop_weight(m, which, kind, a, b, T);
                }
            /* Y[t1 t2 t3 t4] = sum_{l1 l2} (...) */
            for (int t1 = 0; t1 < ns; t1++)
                for (int t2 = 0; t2 < ns; t2++)
                    for (int t3 = 0; t3 < ns; t3++)
                        for (int t4 = 0; t4 < ns; t4++) {
                            cplx y = 0.0;
                            for (int l1 = 0; l1 < ns; l1++)
                                for (int l2 = 0; l2 < ns; l2++) {
                                    cplx left = U1[t1 * ns + l1] * conj(U1[t3 * ns + l1]);
                                    cplx right = (which == 0) ? U2[t2 * ns + l2] * conj(U2[t4 * ns + l2])
                                                              : conj(U2[t2 * ns + l2]) * U2[t4 * ns + l2];
                                    y += left * w[l1 * ns + l2] * right;
                                }
                            int a, b;
                            if (which == 0) { a = t2 * ns + t1; b = t4 * ns + t3; }
                            else            { a = t1 * ns + t2; b = t3 * ns + t4; }
                            Y[a * ns2 + b] = y;
                        }
            for (int d = 0; d < nd; d++) {
                cplx ph = ph_tab[((size_t)qx * Lf + qy) * nd + d];
                cplx *o = acc + (size_t)d * ns4;
                for (int i = 0; i < ns4; i++) o[i] += ph * Y[i];
            }
        }
    for (size_t i = 0; i < (size_t)nd * ns4; i++) acc[i] /= (double)Nk;
    free(Y); free(w);
}

/* e^{-i q.(R1-R2)} for every fine q and bond difference (depends on q only) */
static cplx *loop_phase_table(const or_model *m, const int *dl, int nd)
{
    int Lf = m->Lq * m->nc;
    cplx *ph_tab = malloc(sizeof(cplx) * (size_t)Lf * Lf * nd);
    for (int qx = 0; qx < Lf; qx++)
        for (int qy = 0; qy < Lf; qy++)
            for (int d = 0; d < nd; d++)
                ph_tab[((size_t)qx * Lf + qy) * nd + d] = conj(lattice_phase((long)qx * dl[2 * d] + (long)qy * dl[2 * d + 1], Lf));
    return ph_tab;
}

/*
 * which = 0 (particle-particle, s on the coarse mesh):
 *   [L^-_{t1t2t3t4}(s)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)}
 *        sum_{l1 l2} U_{t1 l1}(s-q) U*_{t3 l1}(s-q) w^-_{l1 l2}(s-q, q) U_{t2 l2}(q) U*_{t4 l2}(q)
 * which = 1 (crossed particle-hole, u on the coarse mesh):
 *   [L^+_{t1t2t3t4}(u)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)}
 *        sum_{l1 l2} U_{t1 l1}(q) U*_{t3 l1}(q) w^+_{l1 l2}(q, q-u) U*_{t2 l2}(q-u) U_{t4 l2}(q-u)
 * kind = 0: w = the flowing loop at scale T (d/dT F, Eq. def_lmp with chi = 1 and Lambda = T), or at
 *           Lambda with the momentum-shell regulator (d/dLambda [chi chi] F, see loop_weight)
 * kind = 1: w = F itself, or chi chi F (the bubbles, used only by the closed-form pins).
 * Output Lc[q][d][a][b] in the matrix pair order given in the file header.
 */
void or_loops(const or_model *m, const double *E, const double *Uin, double T, int which, int kind,
              double *Lc_out)
{
    int ns2 = m->ns * m->ns, ns4 = ns2 * ns2, Nq = m->Lq * m->Lq;
    int dl[2 * 4096];
    int nd = or_delta_list(m, dl);
    cplx *ph_tab = loop_phase_table(m, dl, nd);
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < Nq; s++)
        loops_one(m, E, (const cplx *)Uin, T, which, kind, s, nd, ph_tab, (cplx *)Lc_out + (size_t)s * nd * ns4);
    free(ph_tab);
}

/* Same loops for a list of n transfer momenta only: out[n][nd][ns^2][ns^2]. */
void or_loops_at(const or_model *m, const double *E, const double *Uin, double T, int which, int kind, int n,
                 const int *s_list, double *out)
{
    int ns2 = m->ns * m->ns, ns4 = ns2 * ns2;
    int dl[2 * 4096];
    int nd = or_delta_list(m, dl);
    cplx *ph_tab = loop_phase_table(m, dl, nd);
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; i++)
        loops_one(m, E, (const cplx *)Uin, T, which, kind, s_list[i], nd, ph_tab, (cplx *)out + (size_t)i * nd * ns4);
    free(ph_tab);
}

/* ------------------------------------------------------------------------ */
/* 4.-5. Fourier transform to bonds and the projections                       */
/* ------------------------------------------------------------------------ */

/* X(R) = (1/Nq) sum_u e^{i u.R} X(u)  (Sec. 3.3) for one bond R. */
static void dft_to_bond(const or_model *m, const cplx *X, int Rx, int Ry, cplx *out)
{
    int Lq = m->Lq, Nq = Lq * Lq, M = m->nff * m->ns * m->ns;
    size_t M2 = (size_t)M * M;
    for (size_t i = 0; i < M2; i++) out[i] = 0.0;
    for (int u = 0; u < Nq; u++) {
        cplx ph = lattice_phase((long)(u / Lq) * Rx + (long)(u % Lq) * Ry, Lq);
        const cplx *Xu = X + (size_t)u * M2;
        for (size_t i = 0; i < M2; i++) out[i] += ph * Xu[i];
    }
    for (size_t i = 0; i < M2; i++) out[i] /= (double)Nq;
}

/*
 * A_P(s) and A_C(u) from a state X = (P, C):
 *   P-channel (Eq. sum_P):  P^[V] = P^[V0] + P + P^[V^C] + P^[V^D]
 *     P^[V^C]_{RR'}(s) =  sum_R'' e^{i s.R''} C^{R+R'', R'-R''}_{s1s2s3s4}(R'')            (Eq. proj_PD)
 *     P^[V^D]_{RR'}(s) = -e^{i s.R'} sum_R'' e^{i s.R''} C^{R+R'', -R'-R''}_{s1s2s4s3}(R'')
 *   C-channel:              C^[V] = C^[V0] + C^[V^P] + C + C^[V^D]
 *     C^[V^P]_{RR'}(u) =  sum_R'' e^{i u.R''} P^{R+R'', R'-R''}_{s1s2s3s4}(R'')
 *     C^[V^D]_{RR'}(u) = -sum_R'' e^{i u.R''} C^{R-R'+R'', R''}_{s1s2s4s3}(-R')              (Eq. proj_DC)
 *   V0 is onsite, so its projections are V0 d_{R0} d_{R'0}.
 * R'' runs over lattice vectors modulo Lq; a term whose shifted bond is not
 * (congruent to) a member of the bond set vanishes because the exchange
 * propagators are zero outside it.
 * chmask bit 0 = P flows, bit 1 = C flows; a channel that does not flow is
 * zero and contributes nothing.
 * Returns max |A| over both channels.
 */
typedef struct {
    const or_model *m;
    int chmask, ncls;
    const cplx *P, *C;
    int *cls, *plus, *minus, *negminus, *negcls, *dcidx;
    cplx *Pr, *Cr;
} proj_ctx;

/* The bond classes R'' and the bond look-ups of the projections; Pr, Cr allocated (zero), not yet filled */
static void proj_tables(const or_model *m, int chmask, proj_ctx *c)
{
    int ns2 = m->ns * m->ns, nff = m->nff, M = nff * ns2, Lq = m->Lq;
    size_t M2 = (size_t)M * M;
    c->m = m;
    c->chmask = chmask;
    c->P = c->C = NULL;
    /* R'' classes modulo Lq that can give a non-zero term: differences of two bonds */
    c->cls = malloc(sizeof(int) * 2 * nff * nff);
    int ncls = 0;
    for (int i = 0; i < nff; i++)
        for (int j = 0; j < nff; j++) {
            int x = imod(m->ffR[2 * i] - m->ffR[2 * j], Lq), y = imod(m->ffR[2 * i + 1] - m->ffR[2 * j + 1], Lq);
            int seen = 0;
            for (int k = 0; k < ncls; k++) if (c->cls[2 * k] == x && c->cls[2 * k + 1] == y) { seen = 1; break; }
            if (!seen) { c->cls[2 * ncls] = x; c->cls[2 * ncls + 1] = y; ncls++; }
        }
    c->ncls = ncls;
    c->Pr = calloc((size_t)ncls * M2, sizeof(cplx));
    c->Cr = calloc((size_t)ncls * M2, sizeof(cplx));
    /* bond look-ups (pure bookkeeping of which shifted bonds are in the set) */
    c->plus = malloc(sizeof(int) * nff * ncls);
    c->minus = malloc(sizeof(int) * nff * ncls);
    c->negminus = malloc(sizeof(int) * nff * ncls);
    c->negcls = malloc(sizeof(int) * nff);
    c->dcidx = malloc(sizeof(int) * nff * nff * nff);
    for (int i = 0; i < nff; i++) {
        int Rx = m->ffR[2 * i], Ry = m->ffR[2 * i + 1];
        for (int k = 0; k < ncls; k++) {
            c->plus[i * ncls + k] = ff_index_mod(m, Rx + c->cls[2 * k], Ry + c->cls[2 * k + 1]);
            c->minus[i * ncls + k] = ff_index_mod(m, Rx - c->cls[2 * k], Ry - c->cls[2 * k + 1]);
            c->negminus[i * ncls + k] = ff_index_mod(m, -Rx - c->cls[2 * k], -Ry - c->cls[2 * k + 1]);
        }
        c->negcls[i] = -1;
        for (int k = 0; k < ncls; k++)
            if (c->cls[2 * k] == imod(-Rx, Lq) && c->cls[2 * k + 1] == imod(-Ry, Lq)) c->negcls[i] = k;
        for (int j = 0; j < nff; j++)
            for (int w = 0; w < nff; w++)
                c->dcidx[(i * nff + j) * nff + w] = ff_index_mod(m, Rx - m->ffR[2 * j] + m->ffR[2 * w],
                                                                 Ry - m->ffR[2 * j + 1] + m->ffR[2 * w + 1]);
    }
}

/* Fourier transforms of P and C to every bond class that can occur, plus bond look-ups */
static void proj_prepare(const or_model *m, const double *state, int chmask, proj_ctx *c)
{
    int M = m->nff * m->ns * m->ns, Nq = m->Lq * m->Lq;
    size_t M2 = (size_t)M * M;
    proj_tables(m, chmask, c);
    c->P = (const cplx *)state;
    c->C = c->P + (size_t)Nq * M2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < c->ncls; k++) {
        if (chmask & 1) dft_to_bond(m, c->P, c->cls[2 * k], c->cls[2 * k + 1], c->Pr + (size_t)k * M2);
        if (chmask & 2) dft_to_bond(m, c->C, c->cls[2 * k], c->cls[2 * k + 1], c->Cr + (size_t)k * M2);
    }
}

static void proj_free(proj_ctx *c)
{
    free(c->Pr); free(c->Cr); free(c->cls); free(c->plus); free(c->minus); free(c->negminus); free(c->negcls);
    free(c->dcidx);
}

/* A_P(q) and A_C(q) of one transfer momentum from its own state rows Pq = P(q), Cq = C(q) and the Fourier
 * transforms in c; returns max |A| over both */
static double proj_one(const proj_ctx *c, int q, const cplx *Pq, const cplx *Cq, cplx *AP, cplx *AC)
{
    const or_model *m = c->m;
    int ns = m->ns, ns2 = ns * ns, nff = m->nff, M = nff * ns2, Lq = m->Lq, ncls = c->ncls;
    size_t M2 = (size_t)M * M;
    const cplx *V0 = (const cplx *)m->V0, *V0q = (const cplx *)m->V0q;
    const cplx *Pr = c->Pr, *Cr = c->Cr;
    int i0 = ff_index_mod(m, 0, 0);
    int onP = c->chmask & 1, onC = (c->chmask >> 1) & 1;
    int qx = q / Lq, qy = q % Lq;
    double amax = 0.0;
    for (int iR = 0; iR < nff; iR++)
        for (int iRp = 0; iRp < nff; iRp++) {
            int Rpx = m->ffR[2 * iRp], Rpy = m->ffR[2 * iRp + 1];
            for (int s1 = 0; s1 < ns; s1++)
                for (int s2 = 0; s2 < ns; s2++)
                    for (int s3 = 0; s3 < ns; s3++)
                        for (int s4 = 0; s4 < ns; s4++) {
                            const cplx v0on = (iR == i0 && iRp == i0) ? V0[((s1 * ns + s2) * ns + s3) * ns + s4] : 0.0;
                            /* ---- P channel entry (R,(s1,s2)),(R',(s4,s3)) ---- */
                            if (onP) {
                                size_t row = (size_t)iR * ns2 + s1 * ns + s2, col = (size_t)iRp * ns2 + s4 * ns + s3;
                                cplx v0 = V0q ? V0q[(size_t)q * M2 + row * M + col] : v0on;
                                cplx val = v0 + Pq[row * M + col];
                                if (onC) {
                                    for (int k = 0; k < ncls; k++) {
                                        int Ux = c->cls[2 * k], Uy = c->cls[2 * k + 1];   /* R'' */
                                        int i1 = c->plus[iR * ncls + k];
                                        if (i1 < 0) continue;
                                        int i2 = c->minus[iRp * ncls + k];
                                        if (i2 >= 0) {
                                            cplx ph = lattice_phase((long)qx * Ux + (long)qy * Uy, Lq);
                                            size_t sr = (size_t)i1 * ns2 + s1 * ns + s3, sc = (size_t)i2 * ns2 + s4 * ns + s2;
                                            val += ph * Cr[(size_t)k * M2 + sr * M + sc];
                                        }
                                        int j2 = c->negminus[iRp * ncls + k];
                                        if (j2 >= 0) {
                                            /* C_{s1 s2 s4 s3}: row (s1, s4), column (s3, s2) */
                                            cplx ph2 = lattice_phase((long)qx * (Rpx + Ux) + (long)qy * (Rpy + Uy), Lq);
                                            size_t sr = (size_t)i1 * ns2 + s1 * ns + s4, sc = (size_t)j2 * ns2 + s3 * ns + s2;
                                            val -= ph2 * Cr[(size_t)k * M2 + sr * M + sc];
                                        }
                                    }
                                }
                                AP[row * M + col] = val;
                                if (cabs(val) > amax) amax = cabs(val);
                            }
                            /* ---- C channel entry (R,(s1,s3)),(R',(s4,s2)) ---- */
                            if (onC) {
                                size_t row = (size_t)iR * ns2 + s1 * ns + s3, col = (size_t)iRp * ns2 + s4 * ns + s2;
                                cplx v0 = V0q ? V0q[((size_t)Lq * Lq + q) * M2 + row * M + col] : v0on;
                                cplx val = v0 + Cq[row * M + col];
                                if (onP) {
                                    for (int k = 0; k < ncls; k++) {
                                        int i1 = c->plus[iR * ncls + k], i2 = c->minus[iRp * ncls + k];
                                        if (i1 < 0 || i2 < 0) continue;
                                        cplx ph = lattice_phase((long)qx * c->cls[2 * k] + (long)qy * c->cls[2 * k + 1], Lq);
                                        size_t sr = (size_t)i1 * ns2 + s1 * ns + s2, sc = (size_t)i2 * ns2 + s4 * ns + s3;
                                        val += ph * Pr[(size_t)k * M2 + sr * M + sc];
                                    }
                                }
                                /* D -> C: the Fourier argument is -R', the sum runs over R'' in the bond set */
                                int cm = c->negcls[iRp];
                                for (int i2 = 0; i2 < nff; i2++) {
                                    int i1 = c->dcidx[(iR * nff + iRp) * nff + i2];
                                    if (i1 < 0) continue;
                                    cplx ph = lattice_phase((long)qx * m->ffR[2 * i2] + (long)qy * m->ffR[2 * i2 + 1], Lq);
                                    size_t sr = (size_t)i1 * ns2 + s1 * ns + s4, sc = (size_t)i2 * ns2 + s3 * ns + s2;
                                    val -= ph * Cr[(size_t)cm * M2 + sr * M + sc];
                                }
                                AC[row * M + col] = val;
                                if (cabs(val) > amax) amax = cabs(val);
                            }
                        }
        }
    if (!onP) memset(AP, 0, sizeof(cplx) * M2);
    if (!onC) memset(AC, 0, sizeof(cplx) * M2);
    return amax;
}

double or_project(const or_model *m, const double *state, int chmask, double *Ahat_out)
{
    int M = m->nff * m->ns * m->ns, Nq = m->Lq * m->Lq;
    size_t M2 = (size_t)M * M;
    cplx *AP = (cplx *)Ahat_out, *AC = AP + (size_t)Nq * M2;
    proj_ctx c;
    proj_prepare(m, state, chmask, &c);
    double amax = 0.0;
#pragma omp parallel for schedule(static) reduction(max : amax)
    for (int q = 0; q < Nq; q++) {
        double a = proj_one(&c, q, c.P + (size_t)q * M2, c.C + (size_t)q * M2, AP + (size_t)q * M2, AC + (size_t)q * M2);
        if (a > amax) amax = a;
    }
    proj_free(&c);
    return amax;
}

/* The bare vertex as a state: P(q) and C(q) equal to its projections at every q, the onsite V0 of Sec. 4 in the
 * (R, R') = (0, 0) block, P entry (0,(s1,s2)),(0,(s4,s3)) and C entry (0,(s1,s3)),(0,(s4,s2)) = V0_{s1 s2 s3 s4};
 * out [2][Nq][M][M] complex.  Transformed with or_band_transform it is the bare vertex of the band-basis flow. */
void or_bare_state(const or_model *m, double *out)
{
    int ns = m->ns, ns2 = ns * ns, M = m->nff * ns2, Nq = m->Lq * m->Lq;
    size_t M2 = (size_t)M * M;
    const cplx *V0 = (const cplx *)m->V0;
    cplx *o = (cplx *)out;
    memset(o, 0, sizeof(cplx) * 2 * (size_t)Nq * M2);
    int i0 = ff_index_mod(m, 0, 0);
    for (int q = 0; q < Nq; q++)
        for (int s1 = 0; s1 < ns; s1++)
            for (int s2 = 0; s2 < ns; s2++)
                for (int s3 = 0; s3 < ns; s3++)
                    for (int s4 = 0; s4 < ns; s4++) {
                        cplx v = V0[(((size_t)s1 * ns + s2) * ns + s3) * ns + s4];
                        size_t rP = (size_t)i0 * ns2 + s1 * ns + s2, cP = (size_t)i0 * ns2 + s4 * ns + s3;
                        size_t rC = (size_t)i0 * ns2 + s1 * ns + s3, cC = (size_t)i0 * ns2 + s4 * ns + s2;
                        o[(size_t)q * M2 + rP * M + cP] = v;
                        o[((size_t)Nq + q) * M2 + rC * M + cC] = v;
                    }
}

/* ------------------------------------------------------------------------ */
/* 6. dX/dT = c_X A L A                                                       */
/* ------------------------------------------------------------------------ */

/* Expand the compact loop of one transfer momentum into the M x M matrix
 * L[(R1,a),(R2,b)] = Lc[d(R1-R2)][a][b]. */
static void expand_loop(const or_model *m, const cplx *Lcq, const int *dl, int nd, cplx *Lm)
{
    int ns2 = m->ns * m->ns, M = m->nff * ns2, ns4 = ns2 * ns2;
    for (int i1 = 0; i1 < m->nff; i1++)
        for (int i2 = 0; i2 < m->nff; i2++) {
            int d = delta_index(dl, nd, m->ffR[2 * i1] - m->ffR[2 * i2], m->ffR[2 * i1 + 1] - m->ffR[2 * i2 + 1]);
            for (int a = 0; a < ns2; a++)
                for (int b = 0; b < ns2; b++)
                    Lm[(size_t)(i1 * ns2 + a) * M + i2 * ns2 + b] = Lcq[(size_t)d * ns4 + a * ns2 + b];
        }
}

/* dP/dT(s) = A_P(s) L^-(s) A_P(s) (Eq. RGE_spin);  dC/dT(u) = 2 A_C(u) L^+(u) A_C(u). */
void or_vlv(const or_model *m, const double *Ahat, const double *LcP, const double *LcC, int chmask,
            double *dstate)
{
    int ns2 = m->ns * m->ns, M = m->nff * ns2, ns4 = ns2 * ns2;
    int Nq = m->Lq * m->Lq;
    size_t M2 = (size_t)M * M;
    int dl[2 * 4096];
    int nd = or_delta_list(m, dl);
    memset(dstate, 0, sizeof(cplx) * 2 * Nq * M2);
    for (int ch = 0; ch < 2; ch++) {
        if (!((chmask >> ch) & 1)) continue;
        const cplx *A = (const cplx *)Ahat + (size_t)ch * Nq * M2;
        const cplx *Lc = (const cplx *)(ch == 0 ? LcP : LcC);
        cplx *D = (cplx *)dstate + (size_t)ch * Nq * M2;
        double cx = (ch == 0) ? 1.0 : 2.0;
#pragma omp parallel for schedule(dynamic, 1)
        for (int q = 0; q < Nq; q++) {
            cplx *Lm = malloc(sizeof(cplx) * M2), *Tm = malloc(sizeof(cplx) * M2);
            expand_loop(m, Lc + (size_t)q * nd * ns4, dl, nd, Lm);
            const cplx *Aq = A + (size_t)q * M2;
            for (int i = 0; i < M; i++)
                for (int j = 0; j < M; j++) {
                    cplx s = 0.0;
                    for (int k = 0; k < M; k++) s += Aq[(size_t)i * M + k] * Lm[(size_t)k * M + j];
                    Tm[(size_t)i * M + j] = s;
                }
            for (int i = 0; i < M; i++)
                for (int j = 0; j < M; j++) {
                    cplx s = 0.0;
                    for (int k = 0; k < M; k++) s += Tm[(size_t)i * M + k] * Aq[(size_t)k * M + j];
                    D[(size_t)q * M2 + (size_t)i * M + j] = cx * s;
                }
            free(Lm); free(Tm);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 8. Band basis (Sec. 3.4: Eqs. trafo_P, mat_trafo_P, mat_trafo_D)            */
/* ------------------------------------------------------------------------ */

/* The transformation matrices, from their definitions with f_R(k) = e^{-ik.R} and N = N_k (fine mesh):
 *   U^{RR'}_{s1 s2 n1 n2}(s) = (1/N) sum_k f_R(k) f*_R'(k) U_{s1 n1}(s - k) U_{s2 n2}(k)
 *   X^{RR'}_{s1 s2 n1 n2}(u) = (1/N) sum_k f_R(k) f*_R'(k) U_{s1 n1}(k) U*_{s2 n2}(k - u)
 * and the exchange propagators in the band basis
 *   P_band(s) = sum_sigma [U_{s2 s1 n2 n1}(s)]^dagger P(s) U_{s3 s4 n3 n4}(s)      (Eq. mat_trafo_P)
 *   C_band(u) = sum_sigma [X_{s1 s3 n1 n3}(u)]^dagger C(u) X_{s4 s2 n4 n2}(u)      (Eq. mat_trafo_D)
 * in the layouts of the orbital matrices (P: row (R,(n1,n2)), col (R',(n4,n3)); C: row (R,(n1,n3)),
 * col (R',(n4,n2))).  As M x M matrices, T[(R1,(a,b)),(R,(c,d))] = U^{R1 R}_{b a d c}(s) for P and
 * X^{R1 R}_{a b c d}(u) for C, and the band matrices are T^dagger X T.  Ub[k][sigma][n] are the
 * eigenvectors to use (the band basis depends on their gauge). */
void or_band_transform(const or_model *m, const double *Ub_in, const double *state, double *out)
{
    int ns = m->ns, ns2 = ns * ns, nff = m->nff, M = nff * ns2;
    int Lq = m->Lq, nc = m->nc, Lf = Lq * nc, Nk = Lf * Lf, Nq = Lq * Lq;
    const cplx *Ub = (const cplx *)Ub_in;
    const cplx *X = (const cplx *)state;
    cplx *Y = (cplx *)out;
    for (int ch = 0; ch < 2; ch++) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int s = 0; s < Nq; s++) {
            int sx = (s / Lq) * nc, sy = (s % Lq) * nc;
            cplx *T = calloc((size_t)M * M, sizeof(cplx));
            cplx *W = calloc((size_t)M * M, sizeof(cplx));
            for (int i1 = 0; i1 < nff; i1++)
                for (int i = 0; i < nff; i++) {
                    int Dx = m->ffR[2 * i1] - m->ffR[2 * i], Dy = m->ffR[2 * i1 + 1] - m->ffR[2 * i + 1];
                    for (int kx = 0; kx < Lf; kx++)
                        for (int ky = 0; ky < Lf; ky++) {
                            cplx ph = conj(lattice_phase((long)kx * Dx + (long)ky * Dy, Lf));   /* f_R1 f*_R */
                            int k = kx * Lf + ky;
                            int k2 = ch == 0 ? imod(sx - kx, Lf) * Lf + imod(sy - ky, Lf)      /* s - k */
                                             : imod(kx - sx, Lf) * Lf + imod(ky - sy, Lf);     /* k - u */
                            for (int a = 0; a < ns; a++)
                                for (int b = 0; b < ns; b++)
                                    for (int c = 0; c < ns; c++)
                                        for (int d = 0; d < ns; d++) {
                                            cplx v = ch == 0 ? Ub[(size_t)k2 * ns2 + b * ns + d] * Ub[(size_t)k * ns2 + a * ns + c]
                                                             : Ub[(size_t)k * ns2 + a * ns + c] * conj(Ub[(size_t)k2 * ns2 + b * ns + d]);
                                            T[(size_t)(i1 * ns2 + a * ns + b) * M + i * ns2 + c * ns + d] += ph * v / (double)Nk;
                                        }
                        }
                }
            const cplx *Xs = X + ((size_t)ch * Nq + s) * M * M;
            cplx *Ys = Y + ((size_t)ch * Nq + s) * M * M;
            for (int r = 0; r < M; r++)          /* W = X T */
                for (int c = 0; c < M; c++) {
                    cplx acc = 0.0;
                    for (int j = 0; j < M; j++) acc += Xs[(size_t)r * M + j] * T[(size_t)j * M + c];
                    W[(size_t)r * M + c] = acc;
                }
            for (int r = 0; r < M; r++)          /* Y = T^dagger W */
                for (int c = 0; c < M; c++) {
                    cplx acc = 0.0;
                    for (int j = 0; j < M; j++) acc += conj(T[(size_t)j * M + r]) * W[(size_t)j * M + c];
                    Ys[(size_t)r * M + c] = acc;
                }
            free(T);
            free(W);
        }
    }
}

/* One right-hand side dX/dT at temperature T.  Ahat_out may be NULL. Returns max |A|. */
double or_rhs(const or_model *m, const double *E, const double *U, double T, const double *state,
              int chmask, double *dstate, double *Ahat_out)
{
    int ns2 = m->ns * m->ns, M = m->nff * ns2, ns4 = ns2 * ns2, Nq = m->Lq * m->Lq;
    size_t M2 = (size_t)M * M;
    int dl[2 * 4096];
    int nd = or_delta_list(m, dl);
    double *LcP = calloc((size_t)Nq * nd * ns4 * 2, sizeof(double));
    double *LcC = calloc((size_t)Nq * nd * ns4 * 2, sizeof(double));
    double *A = Ahat_out ? Ahat_out : malloc(sizeof(double) * 2 * 2 * Nq * M2);
    if (chmask & 1) or_loops(m, E, U, T, 0, 0, LcP);
    if (chmask & 2) or_loops(m, E, U, T, 1, 0, LcC);
    double amax = or_project(m, state, chmask, A);
    or_vlv(m, A, LcP, LcC, chmask, dstate);
    free(LcP); free(LcC);
    if (!Ahat_out) free(A);
    return amax;
}

/* dX/dT at the n listed transfer momenta from the projection context c (Fourier transforms and bond
 * look-ups) and the momenta's own state rows: P(s_list[i]) at Prows + i Mrow_stride, C likewise:
 * loops at the listed momenta, the projections, then c_X A L A with c_P = 1, c_C = 2.  out [2][n][M][M]. */
static void rhs_rows(const or_model *m, const double *E, const double *U, double T, const proj_ctx *c,
                     const cplx *Prows, const cplx *Crows, int n, const int *s_list, int chmask, double *out)
{
    int ns2 = m->ns * m->ns, M = m->nff * ns2, ns4 = ns2 * ns2;
    size_t M2 = (size_t)M * M;
    int dl[2 * 4096];
    int nd = or_delta_list(m, dl);
    cplx *Lp = calloc((size_t)n * nd * ns4, sizeof(cplx)), *Lcc = calloc((size_t)n * nd * ns4, sizeof(cplx));
    if (chmask & 1) or_loops_at(m, E, U, T, 0, 0, n, s_list, (double *)Lp);
    if (chmask & 2) or_loops_at(m, E, U, T, 1, 0, n, s_list, (double *)Lcc);
    cplx *o = (cplx *)out;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; i++) {
        cplx *AP = malloc(sizeof(cplx) * M2), *AC = malloc(sizeof(cplx) * M2);
        cplx *Lm = malloc(sizeof(cplx) * M2), *Tm = malloc(sizeof(cplx) * M2);
        proj_one(c, s_list[i], Prows + (size_t)i * M2, Crows + (size_t)i * M2, AP, AC);
        for (int ch = 0; ch < 2; ch++) {
            cplx *D = o + ((size_t)ch * n + i) * M2;
            if (!((chmask >> ch) & 1)) { memset(D, 0, sizeof(cplx) * M2); continue; }
            const cplx *A = ch == 0 ? AP : AC;
            expand_loop(m, (ch == 0 ? Lp : Lcc) + (size_t)i * nd * ns4, dl, nd, Lm);
            double cx = ch == 0 ? 1.0 : 2.0;
            for (int r = 0; r < M; r++)
                for (int col = 0; col < M; col++) {
                    cplx sacc = 0.0;
                    for (int k = 0; k < M; k++) sacc += A[(size_t)r * M + k] * Lm[(size_t)k * M + col];
                    Tm[(size_t)r * M + col] = sacc;
                }
            for (int r = 0; r < M; r++)
                for (int col = 0; col < M; col++) {
                    cplx sacc = 0.0;
                    for (int k = 0; k < M; k++) sacc += Tm[(size_t)r * M + k] * A[(size_t)k * M + col];
                    D[(size_t)r * M + col] = cx * sacc;
                }
        }
        free(AP); free(AC); free(Lm); free(Tm);
    }
    free(Lp); free(Lcc);
}

/* dX/dT for a list of n transfer momenta only (a bounded sample of one right-hand side):
 * out [2][n][M][M].  Same steps as or_rhs, restricted to the listed momenta where possible
 * (the Fourier transform always runs over the whole mesh). */
void or_rhs_at(const or_model *m, const double *E, const double *U, double T, const double *state, int chmask,
               int n, const int *s_list, double *out)
{
    int M = m->nff * m->ns * m->ns, Nq = m->Lq * m->Lq;
    size_t M2 = (size_t)M * M;
    proj_ctx c;
    proj_prepare(m, state, chmask, &c);
    /* the listed momenta's own rows, in list order */
    cplx *rows = malloc(sizeof(cplx) * 2 * (size_t)(n > 0 ? n : 1) * M2);
    for (int i = 0; i < n; i++) {
        memcpy(rows + (size_t)i * M2, c.P + (size_t)s_list[i] * M2, sizeof(cplx) * M2);
        memcpy(rows + ((size_t)n + i) * M2, c.C + (size_t)s_list[i] * M2, sizeof(cplx) * M2);
    }
    (void)Nq;
    rhs_rows(m, E, U, T, &c, rows, rows + (size_t)n * M2, n, s_list, chmask, out);
    free(rows);
    proj_free(&c);
}

/* ------------------------------------------------------------------------ */
/* 6b. The right-hand side with the transfer momenta split into shards        */
/* ------------------------------------------------------------------------ */
/* A shard is a list of n transfer momenta with their own rows of the state, state_local [2][n][M][M].  The
 * only quantity that couples momenta is the Fourier transform of Sec. 3.3, a sum over the whole mesh: each
 * shard forms its part over its own momenta, the parts are summed (an all-reduce), and each shard finishes
 * its own rows from the sum. */

/* Bond classes R'' (mod Lq) of the transforms, [ncls][2], in the order of the xr arrays below; returns ncls */
int or_shard_classes(const or_model *m, int *cls_out)
{
    proj_ctx c;
    proj_tables(m, 3, &c);
    for (int k = 0; k < c.ncls; k++) { cls_out[2 * k] = c.cls[2 * k]; cls_out[2 * k + 1] = c.cls[2 * k + 1]; }
    int n = c.ncls;
    proj_free(&c);
    return n;
}

/* xr [2][ncls][M][M] = (1/Nq) sum_i e^{i q_i.R''} X_local[ch][i] over the listed momenta q_i */
void or_shard_transform(const or_model *m, const double *state_local, int n, const int *q_list, int chmask, double *xr)
{
    int M = m->nff * m->ns * m->ns, Lq = m->Lq, Nq = Lq * Lq;
    size_t M2 = (size_t)M * M;
    proj_ctx c;
    proj_tables(m, chmask, &c);
    const cplx *X = (const cplx *)state_local;
    cplx *o = (cplx *)xr;
    memset(o, 0, sizeof(cplx) * 2 * (size_t)c.ncls * M2);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < c.ncls; k++)
        for (int ch = 0; ch < 2; ch++) {
            if (!((chmask >> ch) & 1)) continue;
            cplx *dst = o + ((size_t)ch * c.ncls + k) * M2;
            for (int i = 0; i < n; i++) {
                int u = q_list[i];
                cplx ph = lattice_phase((long)(u / Lq) * c.cls[2 * k] + (long)(u % Lq) * c.cls[2 * k + 1], Lq);
                const cplx *Xu = X + ((size_t)ch * n + i) * M2;
                for (size_t e = 0; e < M2; e++) dst[e] += ph * Xu[e];
            }
            for (size_t e = 0; e < M2; e++) dst[e] /= (double)Nq;
        }
    proj_free(&c);
}

/* dX/dT at the listed momenta from their own rows and the summed transforms xr: out_local [2][n][M][M] */
void or_shard_finish(const or_model *m, const double *E, const double *U, double T, const double *state_local, int n,
                     const int *q_list, const double *xr, int chmask, double *out_local)
{
    int M = m->nff * m->ns * m->ns;
    size_t M2 = (size_t)M * M;
    proj_ctx c;
    proj_tables(m, chmask, &c);
    memcpy(c.Pr, xr, sizeof(cplx) * (size_t)c.ncls * M2);
    memcpy(c.Cr, (const cplx *)xr + (size_t)c.ncls * M2, sizeof(cplx) * (size_t)c.ncls * M2);
    const cplx *X = (const cplx *)state_local;
    rhs_rows(m, E, U, T, &c, X, X + (size_t)n * M2, n, q_list, chmask, out_local);
    proj_free(&c);
}

/* ------------------------------------------------------------------------ */
/* 7. Dormand-Prince 5(4) flow in x = ln T                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double T0, T_end, rtol, atol, h0, stop;
    int chmask, max_steps;
    int fixed_n;          /* > 0: classic RK4 with this many equal steps in ln T (no control) */
} or_flow_opts;

typedef struct {
    double Tc;            /* interpolated critical scale, or T_end if no crossing */
    int crossed;
    int n_steps, n_reject, n_rhs;
    double amax;          /* max |A| at the last accepted state */
    double T_last;
} or_flow_result;

static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0},
    {1.0 / 5},
    {3.0 / 40, 9.0 / 40},
    {44.0 / 45, -56.0 / 15, 32.0 / 9},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
    {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double DP_B[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0};
static const double DP_BS[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                                187.0 / 2100, 1.0 / 40};

/* f(x, y) = T dy/dT at T = e^x */
static double flow_f(const or_model *m, const double *E, const double *U, double x, const double *y,
                     int chmask, double *out, size_t n)
{
    double T = exp(x);
    double amax = or_rhs(m, E, U, T, y, chmask, out, NULL);
    for (size_t i = 0; i < n; i++) out[i] *= T;
    return amax;
}

/* Integrates the state (initially zero, Eqs. def_VP.. at Lambda_0) from T0 down to T_end or
 * until max|A| exceeds opts->stop.  state_out [2][Nq][M][M] complex receives the last
 * accepted state. */
int or_flow(const or_model *m, const double *E, const double *U, const or_flow_opts *o, double *state_out,
            or_flow_result *res)
{
    int M = m->nff * m->ns * m->ns, Nq = m->Lq * m->Lq;
    size_t n = (size_t)2 * 2 * Nq * M * M;   /* doubles */
    double *y = state_out, *k[7], *yt = malloc(sizeof(double) * n), *yn = malloc(sizeof(double) * n);
    for (int i = 0; i < 7; i++) k[i] = malloc(sizeof(double) * n);
    memset(y, 0, sizeof(double) * n);
    memset(res, 0, sizeof(*res));
    double x = log(o->T0), xend = log(o->T_end);
    double amax_prev = 0.0, x_prev = x;

    if (o->fixed_n > 0) {
        /* classic RK4, fixed steps: used by the brute-force comparison */
        double h = (xend - x) / o->fixed_n;
        static const double a4[4] = {0.0, 0.5, 0.5, 1.0}, b4[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
        for (int st = 0; st < o->fixed_n; st++) {
            for (int j = 0; j < 4; j++) {
                for (size_t i = 0; i < n; i++) yt[i] = y[i] + (j ? a4[j] * h * k[j - 1][i] : 0.0);
                double a = flow_f(m, E, U, x + a4[j] * h, yt, o->chmask, k[j], n);
                if (j == 0) res->amax = a;
                res->n_rhs++;
            }
            for (size_t i = 0; i < n; i++) y[i] += h * (b4[0] * k[0][i] + b4[1] * k[1][i] + b4[2] * k[2][i] + b4[3] * k[3][i]);
            x += h;
            res->n_steps++;
        }
        res->T_last = exp(x);
        res->Tc = res->T_last;
        free(yt); free(yn); for (int i = 0; i < 7; i++) free(k[i]);
        return 0;
    }

    double h = o->h0;
    amax_prev = flow_f(m, E, U, x, y, o->chmask, k[0], n);
    res->n_rhs++;
    res->amax = amax_prev;
    int status = 0;
    /* max|A| above the stop value already at T0: the flow is critical before its first step, Lambda_c = T0 */
    if (amax_prev > o->stop) {
        res->crossed = 1;
        res->Tc = exp(x);
    }
    while (!res->crossed && res->n_steps < o->max_steps) {
        if (x + h < xend) h = xend - x;
        for (int j = 1; j < 7; j++) {
            for (size_t i = 0; i < n; i++) {
                double acc = 0.0;
                for (int l = 0; l < j; l++) acc += DP_A[j][l] * k[l][i];
                yt[i] = y[i] + h * acc;
            }
            if (j == 6) memcpy(yn, yt, sizeof(double) * n);
            double a = flow_f(m, E, U, x + DP_C[j] * h, yt, o->chmask, k[j], n);
            res->n_rhs++;
            if (j == 6) res->amax = a;   /* provisional: max|A| at the candidate state */
        }
        double amax_new = res->amax;
        /* error norm over complex entries */
        double err = 0.0;
        for (size_t i = 0; i < n; i += 2) {
            double er = 0.0, ei = 0.0;
            for (int l = 0; l < 7; l++) {
                double e = DP_B[l] - DP_BS[l];
                er += e * k[l][i]; ei += e * k[l][i + 1];
            }
            double ea = fabs(h) * sqrt(er * er + ei * ei);
            double ya = sqrt(y[i] * y[i] + y[i + 1] * y[i + 1]);
            double yb = sqrt(yn[i] * yn[i] + yn[i + 1] * yn[i + 1]);
            double sc = o->atol + o->rtol * (ya > yb ? ya : yb);
            double r = ea / sc;
            if (r > err) err = r;
        }
        if (!isfinite(err)) { status = 2; break; }
        if (err <= 1.0) {
            x_prev = x;
            x += h;
            memcpy(y, yn, sizeof(double) * n);
            memcpy(k[0], k[6], sizeof(double) * n);
            res->n_steps++;
            double fac = (err > 0) ? 0.9 * pow(err, -0.2) : 5.0;
            if (fac > 5.0) fac = 5.0;
            if (fac < 0.2) fac = 0.2;
            if (amax_new > o->stop) {
                double t = (o->stop - amax_prev) / (amax_new - amax_prev);
                res->Tc = exp(x_prev + t * (x - x_prev));
                res->crossed = 1;
                break;
            }
            amax_prev = amax_new;
            if (x <= xend + 1e-14) break;
            h *= fac;
        } else {
            res->n_reject++;
            double fac = 0.9 * pow(err, -0.2);
            if (fac < 0.2) fac = 0.2;
            if (fac > 1.0) fac = 1.0;
            h *= fac;
            res->amax = amax_prev;
        }
    }
    if (!res->crossed) res->Tc = exp(x);
    res->T_last = exp(x);
    res->amax = res->crossed ? res->amax : amax_prev;
    free(yt); free(yn); for (int i = 0; i < 7; i++) free(k[i]);
    return status;
}
