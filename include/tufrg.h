/*
 * tufrg.h -- C ABI of the GB300 (sm_103a) truncated-unity fRG right-hand side.
 *
 * Method: Schober, Ehrlich, Reckling, Honerkamp, "Truncated-unity functional
 * renormalization group for multiband systems with spin-orbit coupling".
 * The library evaluates the channel-decomposed flow of the exchange
 * propagators P(s) and C(u) in the orbital (spin) basis:
 *
 *   dP/dT(s) = A_P(s) L^-(s) A_P(s)        (Sec. 4.2, Eq. RGE_spin)
 *   dC/dT(u) = 2 A_C(u) L^+(u) A_C(u)      (orbital form of Sec. 3.1, Eq. rge_Dmat)
 *
 * with A_X the projected vertex of Sec. 3.3 (Eq. sum_P and the four gathers
 * Eq. proj_PD ... Eq. proj_DC) and L^- / L^+ the loop matrices of Eqs.
 * loopminus / loopplus dressed into the orbital basis (Eq. loop_orbital).
 * The flow parameter is the temperature by default: Lambda = T, the regulator
 * chi = 1, so the single-scale loops of Eq. def_lmp are d/dT of the bubbles
 * F^-/F^+ (Eqs. disc_2a, disc_2b).  With the momentum-shell regulator
 * (TUFRG_REG_MOMENTUM_SHELL below) the flow parameter is Lambda itself and the
 * loops are d/dLambda [chi chi] F^-/+ at a fixed temperature; every argument
 * named T below is then Lambda, and d/dT reads d/dLambda.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im) doubles (C99 double complex).
 * - Square lattice; Bloch Hamiltonian H(k)[t][t'] = sum_R t_R[t][t'] e^{i k.R}.
 * - Coarse (transfer) mesh Lq x Lq, index q = qx*Lq + qy, q = 2 pi (qx,qy)/Lq.
 *   Fine (loop) mesh Lf = Lq*nc, index k = kx*Lf + ky.
 * - Bonds (form factors f_R(k) = e^{-i k.R}, Sec. 2): n_ff vectors, ff_R[0] = (0,0),
 *   pairwise distinct modulo Lq.  M = n_ff * n_s^2.
 * - State / derivative / projected vertex: X[2][Nq][M][M], channel 0 = P,
 *   channel 1 = C, row-major M x M per transfer momentum:
 *     P row (R,(s1,s2)), column (R',(s4,s3)) holds P^{RR'}_{s1 s2 s3 s4}(s)
 *     C row (R,(s1,s3)), column (R',(s4,s2)) holds C^{RR'}_{s1 s2 s3 s4}(u)
 *   where (a,b) = a*n_s + b and the R index is the position in ff_R.  In these
 *   layouts the flow equations above are plain matrix products and
 *   hermiticity (Sec. 2, item 3) is matrix hermiticity.
 * - Compact loops: Lc[Nq][n_delta][n_s^2][n_s^2], delta indexing the sorted
 *   (by dx, then dy) list of distinct bond differences R1 - R2 (tufrg_deltas),
 *     P: Lc[q][d][(t2,t1)][(t4,t3)] = [L^-_{t1t2t3t4}(q)]_{R1R2}, R1-R2 = delta_d
 *     C: Lc[q][d][(t1,t2)][(t3,t4)] = [L^+_{t1t2t3t4}(q)]_{R1R2}
 *   so the M x M loop matrix is L[(R1,a),(R2,b)] = Lc[q][d(R1-R2)][a][b].
 * - Every call is stream-ordered on the stream given to tufrg_init_model and
 *   returns a status; no call throws, aborts or exits.  On error the outputs
 *   are unspecified and tufrg_last_error() describes the cause.  A call that
 *   fails on a CUDA runtime call consumes that error (cudaGetLastError), so
 *   it is not left pending for the caller's next launch check; tufrg_init_model
 *   also discards an error left pending by the caller's earlier runtime calls.
 * - Device pointers (prefix d_) must be device memory of the current device
 *   with the documented size, owned by the caller; host pointers (h_) are
 *   host memory owned by the caller.  Descriptors are copied at init.
 */
#ifndef TUFRG_H
#define TUFRG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TUFRG_OK = 0,
    TUFRG_EINVAL = 1,      /* invalid argument or descriptor */
    TUFRG_ENOMEM = 2,      /* device or host allocation failed */
    TUFRG_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    TUFRG_ENONFINITE = 4,  /* a right-hand side or error norm was not finite */
    TUFRG_ENOTCONV = 5,    /* step size underflow or step limit in the flow */
    TUFRG_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
    TUFRG_EFALLBACK = 7,   /* surrogate rejected, direct loops used (informational) */
    TUFRG_ENOTSUP = 8,     /* configuration not supported by the library */
    TUFRG_ETOOBIG = 9      /* problem larger than the fixed scratch of tufrg_loops_noalloc, or projection
                              tables beyond 2^31 entries at init */
} tufrg_status;

/* TUFRG_FP64: every step in FP64.  TUFRG_SPLIT32: FP32 loop sums, FP32 Fourier transform and gathers,
 * FP32-accurate products; the state and its update stay FP64. */
enum { TUFRG_FP64 = 0, TUFRG_SPLIT32 = 1 };
/* Backend of the V.L.V products on the split path: tensor cores (tcgen05, 3xTF32, FP32 accumulation in
 * tensor memory) or FP32 CUDA cores; AUTO times both on the model's sizes at init and keeps the faster.
 * The timed choice is made once per shape in the process (device, precision and sizes) and reused by
 * later models of that shape, so that equal models take equal paths and give equal results. */
enum { TUFRG_PRODUCTS_AUTO = 0, TUFRG_PRODUCTS_TC = 1, TUFRG_PRODUCTS_SIMT = 2 };
enum { TUFRG_CH_P = 1, TUFRG_CH_C = 2 };

typedef struct tufrg_model tufrg_model;   /* opaque; owns all of its device memory */

/* Model descriptor (host memory, copied by tufrg_init_model). */
typedef struct {
    int n_s;               /* spin-orbitals N_s (1..8) */
    int n_hop;             /* number of hopping matrices */
    const int *hop_R;      /* [n_hop][2] lattice vectors R */
    const double *hop_t;   /* [n_hop][n_s][n_s] complex t_R; H(k) must be Hermitian */
    double mu;             /* chemical potential, used when filling <= 0 */
    double filling;        /* > 0: electrons per site; mu is bisected at T_mu and held fixed */
    double T_mu;           /* temperature of the mu bisection */
    const double *V0;      /* [n_s]^4 complex onsite antisymmetric initial vertex V0[s1][s2][s3][s4] */
    int n_ff;              /* bonds (form factors) */
    const int *ff_R;       /* [n_ff][2], ff_R[0] must be (0,0), distinct modulo Lq */
    int Lq;                /* coarse transfer mesh Lq x Lq (>= 2) */
    int nc;                /* fine points per coarse cell per direction (>= 1) */
    int precision;         /* TUFRG_FP64 or TUFRG_SPLIT32 (see above) */
    int products;          /* TUFRG_PRODUCTS_AUTO / _TC / _SIMT (split path only) */
    int symmetry;          /* TUFRG_SYMMETRY_AUTO or TUFRG_SYMMETRY_OFF (see below) */
    int regulator;         /* TUFRG_REG_TEMPERATURE or TUFRG_REG_MOMENTUM_SHELL (see below) */
    double T_reg;          /* momentum shell: temperature of the Fermi functions in the bubbles (> 0) */
    int loops;             /* TUFRG_LOOPS_AUTO / _TC / _SIMT: backend of the multi-orbital loop k-sum (see below) */
    int basis;             /* TUFRG_BASIS_ORBITAL or TUFRG_BASIS_BAND: the single-particle basis of the flow (below) */
} tufrg_model_desc;

/* Single-particle basis of the exchange propagators and of the flow (Sec. 3.2, Sec. 3.4).
 * ORBITAL: states in the orbital (spin) basis, loops of Eq. loop_orbital (the library's default).
 * BAND: the flow in the band basis of the model's eigenvectors U(k), Eqs. rge_Pmat and rge_Dmat: the loops are
 * band-diagonal (Eqs. loopminus, loopplus with the weights of Eqs. disc_2a, disc_2b), and the bare vertex, onsite
 * in the orbital basis, enters through its band-basis projections P^[V0](s) = T_P^dagger P^[V0]_orb T_P and
 * C^[V0](u) = T_C^dagger C^[V0]_orb T_C (Eqs. mat_trafo_P, mat_trafo_D, the transformation of tufrg_band_basis),
 * which depend on the transfer momentum.  States, loops and right-hand sides are band-basis objects in the
 * layouts of the orbital ones with band indices in place of orbital indices; they depend on the gauge of the
 * eigenvectors.  With the complete bond set the two bases give the same flow (related by the transformation);
 * truncated, the band basis needs more bonds (Sec. 3.4).  Two-band models with M <= 64 (else TUFRG_ENOTSUP); the
 * loop symmetries are not used; no surrogate; tufrg_bands then reports unit eigenvectors. */
enum { TUFRG_BASIS_ORBITAL = 0, TUFRG_BASIS_BAND = 1 };

/* Backend of the loop k-sum of split-precision models with N_s = 6 and at most three non-negative y components
 * of the bond differences (5 or 9 bonds): TC runs the per-column orbital sums as complex 3xTF32 GEMMs on the
 * tensor cores (FP32 accumulation in tensor memory), SIMT as FP32 FMAs on the CUDA cores; AUTO takes TC where it
 * applies.  Every other model uses the CUDA-core kernels whatever the value. */
enum { TUFRG_LOOPS_AUTO = 0, TUFRG_LOOPS_TC = 1, TUFRG_LOOPS_SIMT = 2 };

/* Regulator of the loops (Eq. def_lmp, L = d/dLambda [chi(e1) chi(e2)] F(e1, e2)).
 * TEMPERATURE: the flow scale is the temperature, chi = 1, L = d/dT F(e1, e2; T).
 * MOMENTUM_SHELL: the flow scale is Lambda, chi_Lambda(e) = e^2 / (e^2 + Lambda^2) suppresses a shell of
 * thickness Lambda around the Fermi surfaces, and F is taken at the fixed temperature T_reg.
 * The scale argument of tufrg_loops / tufrg_rhs and the T0 / T_end range of a flow are T or Lambda
 * accordingly; the learned surrogate and tufrg_loops_noalloc support the temperature flow only. */
enum { TUFRG_REG_TEMPERATURE = 0, TUFRG_REG_MOMENTUM_SHELL = 1 };

/* Symmetries of the loop k-sums (split two-band path).  A point operation G of the square lattice
 * (rotations by multiples of 90 degrees, the four mirrors) with a spin unitary U such that every
 * hopping satisfies t_{G R} = U t_R U^dagger maps the band projectors as P_l(G k) = U P_l(k) U^dagger,
 * so both loops obey Lc(G q)[G Delta] = V Lc(q)[Delta] V^dagger (V = U (x) U on the P orbital pair,
 * U (x) U^* on the C pair).  Time reversal, t_R = W t_R^* W^T with W = i sigma_y, gives
 * Lc(-q)[Delta] = V conj(Lc(q)[Delta]) V^dagger with V built from W.  With TUFRG_SYMMETRY_AUTO the
 * operations that hold (U searched among the monomial unitaries) are found at init, the k-sum runs
 * for one momentum per orbit and the others are written from it.  TUFRG_SYMMETRY_OFF sums every q. */
/* For symmetric states (tufrg_rhs with TUFRG_SYMMETRIC_STATE, and every flow) the projections and products can
 * run for the orbit representatives only, and do so whenever the state symmetries hold (AUTO and STATES
 * alike; OFF disables every symmetry).  Both paths are timed at init for tufrg_symmetry_info. */
enum { TUFRG_SYMMETRY_AUTO = 0, TUFRG_SYMMETRY_OFF = 1, TUFRG_SYMMETRY_STATES = 2 };

/* Adaptive flow options (Dormand-Prince 5(4) in x = ln T, from T0 down to T_end; T is Lambda with the
 * momentum-shell regulator). */
typedef struct {
    double T0, T_end;      /* start and end of the flow scale, T0 > T_end > 0 */
    double rtol, atol;     /* error norm max_i |err_i| / (atol + rtol max(|y_i|, |y'_i|)) <= 1 */
    double h0;             /* first step in ln T (negative) */
    double stop;           /* stop when max |A_X(q)| over channels, q, entries exceeds this */
    int channel_mask;      /* TUFRG_CH_P | TUFRG_CH_C */
    int max_steps;         /* accepted + rejected step limit */
} tufrg_flow_opts;

typedef struct {
    double Tc;             /* critical scale (linear interpolation in ln T), or T_last if not crossed */
    int crossed;           /* 1 if max|A| exceeded opts.stop */
    int n_steps, n_reject, n_rhs;
    double amax;           /* max |A| at the last accepted state */
    double T_last;         /* temperature of the last accepted state */
    int lead_channel;      /* 0 = P, 1 = C: channel holding max |A| at the last state */
    int lead_q;            /* transfer momentum index of that maximum */
    double wall_s;         /* host wall time of the flow call */
} tufrg_flow_result;

/* Build the model: copies the descriptor, computes the eigensystem of H(k) on
 * the fine mesh (Sec. 3.1; FP64), bisects mu if requested, builds the bond
 * and projection gather tables (Sec. 3.3) and allocates all work memory.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: TUFRG_EINVAL (bad descriptor, non-Hermitian H, bonds not distinct modulo Lq), TUFRG_ENOTSUP (n_s other
 * than 2, 4, 6), TUFRG_ETOOBIG (projection tables beyond 2^31 entries), TUFRG_ENOMEM (a device allocation, or a
 * host allocation for the tables, failed; every entry point maps a device allocation failure to it), TUFRG_ECUDA,
 * TUFRG_ETIMEOUT (a bounded device-side wait gave up while the products backends were timed).  Ownership: on success and on every failure after the model object was
 * allocated, *out holds it (on failure with the message for tufrg_last_error and whatever device memory was already
 * allocated); the caller releases it with tufrg_free in both cases.  *out is NULL only when out or desc is NULL
 * or the host allocation of the object itself failed. */
tufrg_status tufrg_init_model(const tufrg_model_desc *desc, void *cuda_stream, tufrg_model **out);

/* Release every resource of the model (NULL is ignored). */
void tufrg_free(tufrg_model *m);

/* Human-readable description of the last error on this model ("" if none). */
const char *tufrg_last_error(const tufrg_model *m);

/* Sizes: Nq, M, n_delta (loop bond differences), Nk and the chemical potential in use (host outputs).
 * (tufrg_model_info below also reports the products backend chosen at init.)
 * The host queries below (tufrg_dims, tufrg_model_info, tufrg_loop_momenta, tufrg_deltas,
 * tufrg_gather_table) touch no device memory and return TUFRG_EINVAL for a NULL model; in tufrg_dims and
 * tufrg_model_info any output may be NULL (not written), the others need theirs (tufrg_gather_table: h_out
 * may be NULL to count only; channel must be 0 or 1 and cap >= 0, else TUFRG_EINVAL). */
tufrg_status tufrg_dims(const tufrg_model *m, int *Nq, int *M, int *n_delta, int *Nk, double *mu);

/* Products backend in use on the split path (TUFRG_PRODUCTS_TC or _SIMT; _SIMT for FP64 models)
 * and, when AUTO chose it, the two measured times in milliseconds (else -1). */
tufrg_status tufrg_model_info(const tufrg_model *m, int *products, double *ms_tc, double *ms_simt);

/* Number of transfer momenta whose loop k-sums are evaluated directly (Nq unless loop symmetries
 * reduce them, see TUFRG_SYMMETRY_AUTO). */
tufrg_status tufrg_loop_momenta(const tufrg_model *m, int *n_direct);

/* Loop k-sum backend in use: TUFRG_LOOPS_TC (tensor cores) or TUFRG_LOOPS_SIMT (CUDA cores).
 * Errors: TUFRG_EINVAL for NULL arguments. */
tufrg_status tufrg_loops_info(const tufrg_model *m, int *backend);

/* Launch shape of the loop k-sum: *ky_chunks = the number of k_y ranges each fine-mesh column is split into (the
 * grid's depth; every range ends with a flush of its partial sums), and, for the two-band split path, which times
 * every candidate from 1 to 16 ranges (each range at least 8 rows) at model set-up and keeps the fastest:
 * *n_candidates = their number and h_ms[i] (i < min(n_ms, *n_candidates)) = the measured milliseconds per launch
 * of candidate i, which has i + 1 ranges.  Other paths report their heuristic choice and *n_candidates = 0.
 * The choice is cached per process and model shape, so models of the same shape sum in the same order.
 * Errors: TUFRG_EINVAL for NULL arguments or n_ms < 0 (h_ms may be NULL when n_ms is 0). */
tufrg_status tufrg_loop_tiles(const tufrg_model *m, int *ky_chunks, int *n_candidates, double *h_ms, int n_ms);

/* Tile shape of the tensor-core products (split path): *tile_width = the complex columns per output tile (128-row
 * tiles of NB columns; 0 for FP64 models), and, when the products backend was autotuned (TUFRG_PRODUCTS_AUTO), the
 * timings of the column-tile candidates the autotuner compared: *n_candidates = their number and h_ms[i]
 * (i < min(n_ms, *n_candidates)) the milliseconds of candidate i (i = 0: the widest tiles, at most 112 columns;
 * i = 1: one tile more per matrix).  The tiling does not change any output element's summation order.
 * Errors: TUFRG_EINVAL for NULL arguments or n_ms < 0. */
tufrg_status tufrg_products_tiles(const tufrg_model *m, int *tile_width, int *n_candidates, double *h_ms, int n_ms);

/* Exchange propagators of a state in the band basis of the model's eigenvectors (Sec. 3.4, Eqs. trafo_P,
 * mat_trafo_P, mat_trafo_D): with f_R(k) = e^{-ik.R}, N the fine mesh's k-points and U the eigenvectors of
 * tufrg_bands,
 *   U^{RR'}_{s1 s2 n1 n2}(s) = (1/N) sum_k f_R(k) f*_R'(k) U_{s1 n1}(s - k) U_{s2 n2}(k),
 *   X^{RR'}_{s1 s2 n1 n2}(u) = (1/N) sum_k f_R(k) f*_R'(k) U_{s1 n1}(k) U*_{s2 n2}(k - u),
 *   P_band(s) = sum_sigma [U_{s2 s1 n2 n1}(s)]^dagger P(s) U_{s3 s4 n3 n4}(s),
 *   C_band(u) = sum_sigma [X_{s1 s3 n1 n3}(u)]^dagger C(u) X_{s4 s2 n4 n2}(u).
 * d_state, d_out: [2][Nq][M][M] complex device buffers in the layouts of the orbital matrices with band
 * indices in place of the orbital ones (P: row (R,(n1,n2)), col (R',(n4,n3)); C: row (R,(n1,n3)),
 * col (R',(n4,n2))).  The result depends on the gauge of the eigenvectors.  FP64 models compute in FP64,
 * split models in FP32.  Two-band models with M <= 64 (else TUFRG_ENOTSUP); stream ordered, no host sync. */
tufrg_status tufrg_band_basis(tufrg_model *m, const void *d_state, void *d_out);

/* Form factors of the irreducible representations of the point group C4v (Sec. 2: linear combinations of the plane
 * waves that transform under an irreducible representation).  For a bond set closed under the eight point
 * operations of the square lattice (as integer vectors), the bonds fall into shells (orbits) and each shell's
 * combinations are f_i(k) = sum_R W[i][R] f_R(k), W real orthogonal: h_W [n_ff][n_ff] (row i over the bonds in the
 * order of ff_R), h_labels [n_ff][3] = (shell, irrep, partner) with irrep 0..4 = A1, A2, B1, B2, E (e.g. the nearest-
 * neighbour shell gives the extended s-wave A1, d_{x^2-y^2} B1 and the two p-waves E).  Within an E space (and a
 * repeated irrep of a larger shell) the basis is one orthonormal choice.  Errors: TUFRG_EINVAL (NULL argument),
 * TUFRG_ENOTSUP (bond set not closed under C4v). */
tufrg_status tufrg_form_factors(const tufrg_model *m, double *h_W, int *h_labels);

/* Exchange propagators in the irrep form factors: d_out = (W x 1) X (W x 1)^T per momentum and channel (inverse != 0:
 * W^T in place of W, back to the bonds); d_state, d_out [2][Nq][M][M] complex device buffers (not the same buffer),
 * rows and columns (form factor i, orbital pair) in the layouts of the state.  FP64; stream ordered.
 * Errors: TUFRG_EINVAL, TUFRG_ENOTSUP (bond set not closed under C4v), TUFRG_ECUDA. */
tufrg_status tufrg_irrep_basis(tufrg_model *m, const void *d_state, int inverse, void *d_out);

/* Round n FP64 values at d_in to FP32 at d_out (device buffers, no overlap), to nearest with ties to
 * even: the rounding the split path applies to states, loop data and tables.  Stream ordered on
 * cuda_stream (NULL = legacy default stream).  Errors: TUFRG_EINVAL for NULL buffers with n > 0,
 * TUFRG_ECUDA for a failed launch. */
tufrg_status tufrg_round_f32(const void *d_in, void *d_out, size_t n, void *cuda_stream);

/* Widen n FP32 values at d_in to FP64 at d_out (device buffers, no overlap), exactly (subnormals, signed zeros,
 * infinities and NaN payloads included): the widening the split path applies to its FP32 results.  Stream ordered
 * on cuda_stream (NULL = legacy default stream).  Errors: TUFRG_EINVAL for NULL buffers with n > 0, TUFRG_ECUDA
 * for a failed launch. */
tufrg_status tufrg_widen_f64(const void *d_in, void *d_out, size_t n, void *cuda_stream);

/* Symmetric-state path (TUFRG_SYMMETRIC_STATE): *in_use = 1 when calls that set the flag project and
 * multiply at the orbit representatives only, 0 when they take the general path (the state symmetries
 * do not hold for this model).  *ms_general and *ms_reps are the init-time timings of projections +
 * products of both channels on the two paths in milliseconds (-1 when not measured).
 * Errors: TUFRG_EINVAL for NULL arguments. */
tufrg_status tufrg_symmetry_info(const tufrg_model *m, int *in_use, double *ms_general, double *ms_reps);

/* Host copy of the sorted bond-difference list [n_delta][2] used by the compact loops. */
tufrg_status tufrg_deltas(const tufrg_model *m, int *h_out);

/* Projection gather table of one output channel (0 = P, 1 = C), Sec. 3.3.
 * Each term is 9 int32: iR, iR', kind, R''x, R''y, i1, i2, phase_x, phase_y, where
 * kind 0 = P<-C (Eq. proj_PD), 1 = P<-D, 2 = C<-P, 3 = C<-D (Eq. proj_DC);
 * R'' and the phase vector are reduced modulo Lq into [0, Lq).  The term adds
 * sign * e^{i q.phase} * X_src(R'')[(i1, pair),(i2, pair')] with sign -1 for the
 * D kinds.  Writes at most cap terms, returns the total count in *n_terms. */
tufrg_status tufrg_gather_table(const tufrg_model *m, int channel, int *h_out, int cap, int *n_terms);

/* Eigensystem on the fine mesh (Sec. 3.1, Eq. trafo; computed in FP64 at init): d_E [Nk][n_s] doubles
 * (ascending E, not shifted by mu), d_U [Nk][n_s][n_s] complex, column l the eigenvector of E_l.
 * Errors: TUFRG_EINVAL (NULL argument), TUFRG_ECUDA. */
tufrg_status tufrg_bands(tufrg_model *m, double *d_E, double *d_U);

/* Compact loops d/dT F at temperature T (Eqs. loopminus, loopplus, loop_orbital,
 * fine-mesh direct k-sum).  d_loops: [2][Nq][n_delta][n_s^2][n_s^2] complex; the
 * channels not in channel_mask are left untouched.  Errors: TUFRG_EINVAL (NULL argument, T not positive
 * and finite, channel_mask not a subset of P|C), TUFRG_ECUDA. */
tufrg_status tufrg_loops(tufrg_model *m, double T, int channel_mask, void *d_loops);

/* Projected vertices A_P(s), A_C(u) of a state (Eq. sum_P, Eq. proj_PD, the
 * D->P gather, the P->C gather, Eq. proj_DC).  d_state, d_Ahat: [2][Nq][M][M]
 * complex.  A channel outside channel_mask is treated as zero and its A is
 * zero-filled.  *h_amax (may be NULL) receives max |A| (synchronises).
 * Errors: TUFRG_EINVAL (NULL argument, channel_mask not a subset of P|C), TUFRG_ECUDA. */
tufrg_status tufrg_project(tufrg_model *m, const void *d_state, int channel_mask, void *d_Ahat,
                           double *h_amax);

/* Right-hand side dX/dT of the flow at temperature T (device buffers, no host sync):
 * loops, Fourier transform to bonds, projections, dP/dT = A L^- A, dC/dT = 2 A L^+ A.
 * d_state, d_dstate: [2][Nq][M][M] complex; channels outside the mask get zero.
 * channel_mask may include TUFRG_SYMMETRIC_STATE: the caller asserts that the state has the model's loop
 * symmetries (X(G q) = W X(q) W^dagger, W the bond permutation times the orbital-pair map of the symmetry;
 * every state of a flow from X = 0 has them when the bare vertex does), and projections and products then
 * run for the orbit representatives only, the other momenta being written from them.  For a state without
 * those symmetries the result is wrong; the flag is ignored when the model has no usable symmetry.
 * The second call for a given (d_state, d_dstate, channel_mask) captures the evaluation's launches (after the
 * temperature, which they read from device memory) in a CUDA graph that later calls with the same three replay;
 * the four most recently used triples are kept.  Results are those of direct launches, bit for bit.  On the legacy
 * default stream (not capturable) the graph runs on a private stream ordered after it and before its next work by
 * events.  Calls launch directly while the caller captures the model's stream, while the phases are being timed
 * (tufrg_timing_begin) and with a loop surrogate.
 * Errors: TUFRG_EINVAL (NULL argument, T not positive and finite, bad channel_mask), TUFRG_ECUDA. */
enum { TUFRG_SYMMETRIC_STATE = 4 };
tufrg_status tufrg_rhs(tufrg_model *m, double T, const void *d_state, int channel_mask, void *d_dstate);

/* ------------------------------------------------------------------------------------------
 * The right-hand side split over shards of transfer momenta (one shard per GPU / rank).
 * Loops, projections and products of a transfer momentum need only that momentum, except for the
 * lattice Fourier transform of the exchange propagators to the bond classes R'' (Sec. 3.3, the
 * transform after Eq. zw_1), X(R'') = (1/Nq) sum_u e^{i u.R''} X(u), a sum over the whole transfer mesh.
 * A shard holds the state rows of its own momenta only, in list order: state_local [2][n_q][M][M]
 * complex (channel, list position, layout of tufrg_rhs).  One evaluation is
 *   1. tufrg_rhs_shard_transform: this shard's part of the transforms, d_xr [2][ncls][M][M] complex;
 *   2. the caller sums d_xr over all shards (an all-reduce of 2 ncls M^2 complex numbers, e.g. NCCL);
 *   3. tufrg_rhs_shard_finish: loops at the shard's momenta, projections from the summed transforms,
 *      products: d_dstate_local [2][n_q][M][M], dX/dT of the shard's momenta in list order.
 * With the shards partitioning the mesh, the rows equal those of tufrg_rhs.  h_q_list: n_q distinct
 * momenta in [0, Nq) (host memory); the model keeps full-size work buffers, the shard's rows alone are
 * read and written.  The loops are summed at the listed momenta (the FP64 two-band path sums every
 * momentum); the general (not symmetric-state) path is taken; a model with an attached surrogate is
 * refused (TUFRG_ENOTSUP).  Stream ordered, no host synchronisation beyond the list upload.
 * Errors: TUFRG_EINVAL (NULL argument, bad list, T not positive and finite, bad mask), TUFRG_ENOTSUP,
 * TUFRG_ENOMEM, TUFRG_ECUDA.
 * ------------------------------------------------------------------------------------------ */
/* Number of bond classes ncls of the transforms and, when h_cls is not NULL, the classes [ncls][2] (mod Lq). */
tufrg_status tufrg_shard_classes(const tufrg_model *m, int *ncls, int *h_cls);
tufrg_status tufrg_rhs_shard_transform(tufrg_model *m, const void *d_state_local, int n_q, const int *h_q_list,
                                       int channel_mask, void *d_xr);
tufrg_status tufrg_rhs_shard_finish(tufrg_model *m, double T, const void *d_state_local, int n_q, const int *h_q_list,
                                    const void *d_xr, int channel_mask, void *d_dstate_local);

/* Same right-hand side with host buffers: copies h_state to the device, evaluates,
 * copies dX/dT back into h_dstate and synchronises the stream.  Errors: those of tufrg_rhs, and
 * TUFRG_ETIMEOUT when a bounded device-side wait gave up (the device error flag is read after the sync). */
tufrg_status tufrg_rhs_host(tufrg_model *m, double T, const void *h_state, int channel_mask, void *h_dstate);

/* n right-hand sides from and to host memory with the transfers overlapped: step i reads the state at
 * h_states[i] and writes dX/dT at T[i] to h_dstates[i] (host buffers in the layout of tufrg_rhs, pinned
 * for the copies to overlap; a pointer may repeat).  The host -> device copy of step i + 1 and the
 * device -> host copy of step i - 1 run on two copy streams of the model while step i is evaluated on the
 * model's stream (two device buffers per direction, allocated at the first call).  Returns when every
 * result has arrived.  channel_mask as for tufrg_rhs (TUFRG_SYMMETRIC_STATE included).  Errors as for
 * tufrg_rhs_host; the host buffers are not in use any more when the call returns, also on error. */
tufrg_status tufrg_rhs_host_batch(tufrg_model *m, int n, const double *T, const void *const *h_states, int channel_mask,
                                  void *const *h_dstates);

/* Adaptive flow from X(T0) = 0 (Eqs. def_VP... at Lambda_0) down to T_end or to
 * max|A| > opts->stop.  The Dormand-Prince controller runs on the device: one attempt
 * (six stage right-hand sides, error norm, accept/reject, FSAL commit) is captured once as
 * a CUDA graph and replayed; the host only polls the controller state between attempts.
 * d_state_out (may be NULL): [2][Nq][M][M] complex, the last accepted state.  *res (and d_state_out) are
 * filled on success and on TUFRG_ENOTCONV / TUFRG_ENONFINITE (the state reached so far).  A flow whose
 * max |A| already exceeds opts->stop at T0 (the bare vertex alone) is critical there: crossed = 1, Tc = T0,
 * n_steps = 0, n_rhs = 1.
 * Errors: TUFRG_EINVAL (NULL argument, not T0 > T_end > 0, rtol <= 0, atol < 0, h0 >= 0, channel_mask
 * empty or beyond P|C, max_steps < 1), TUFRG_ENOTCONV (step limit reached or step size underflow),
 * TUFRG_ENONFINITE (non-finite right-hand side or error norm), TUFRG_ETIMEOUT (a bounded device-side wait
 * gave up), TUFRG_ECUDA. */
tufrg_status tufrg_flow(tufrg_model *m, const tufrg_flow_opts *opts, void *d_state_out, tufrg_flow_result *res);

/* Loop k-sum that allocates nothing (no counterpart in the paper; an interface addition).
 *
 * For callers that cannot call cudaMalloc: code that runs where device allocation
 * is forbidden or must go through a host framework's own allocator, and code that
 * must not change the device's memory footprint while it runs.  It computes the
 * same compact loops as tufrg_loops on a TUFRG_SPLIT32 model (N_s = 2, FP32 sums,
 * bond sets whose non-negative bond-difference y components number at most 3, e.g.
 * 5 or 9 bonds), but takes every input from the caller and keeps its scratch (the
 * per-k records and the partial sums) in one file-scope device array of
 * TUFRG_NOALLOC_SCRATCH_BYTES bytes, which every GPU that loads the library holds
 * until the process exits.
 *
 *   Lq, nc          coarse mesh Lq x Lq, nc fine points per cell (Lf = Lq*nc)
 *   d_E             device [Lf*Lf][2] band energies E_l(k), ascending, k = kx*Lf + ky
 *   d_U             device [Lf*Lf][2][2] complex eigenvectors (row orbital, column band),
 *                   e.g. as returned by tufrg_bands
 *   mu, T           chemical potential and temperature (T > 0)
 *   n_ff, h_ffR     host [n_ff][2] bonds, ff_R[0] = (0,0), as in tufrg_model_desc
 *   channel_mask    TUFRG_CH_P | TUFRG_CH_C
 *   d_loops         device [2][Lq*Lq][n_delta][4][4] complex output, layout of tufrg_loops;
 *                   channels outside the mask are left untouched
 *   cuda_stream     stream for all work (NULL = legacy default stream)
 *
 * The scratch must hold Lf*Lf*48 bytes of records plus the partial sums of one
 * channel, Lq*Lq * 2*ceil(Lf/64) * n_dx * n_dy * 128 bytes (n_dx distinct x and n_dy
 * non-negative y components of the bond differences); a larger problem returns
 * TUFRG_ETOOBIG before any work.  Every call made outside stream capture looks
 * up the device address of the scratch with cudaGetSymbolAddress (the device must
 * be current), so a device reset between calls is harmless; a call made while its
 * stream is being captured reuses the address of the last uncaptured call on the
 * device, so make one call before any capture (and again after a device reset);
 * without one it returns TUFRG_ECUDA.  Calls share the
 * scratch: calls that overlap on the GPU (other streams, other threads) race and
 * give wrong results.  Nothing in the scratch needs to start at zero: every record
 * and every partial that is read is first written by the same call.
 * Errors: TUFRG_EINVAL (bad arguments), TUFRG_ENOTSUP (configuration), TUFRG_ETOOBIG,
 * TUFRG_ECUDA (a launch or the symbol look-up failed). */
#define TUFRG_NOALLOC_SCRATCH_BYTES (16u << 20)
tufrg_status tufrg_loops_noalloc(int Lq, int nc, const double *d_E, const double *d_U, double mu, double T, int n_ff,
                                 const int *h_ffR, int channel_mask, void *d_loops, void *cuda_stream);

/* Many independent adaptive flows at once (uneven sizes allowed).  Each model must have been created
 * on its own stream; every flow runs exactly as tufrg_flow would (same device controller, one captured
 * CUDA graph per model per Dormand-Prince attempt), and the attempts of all running flows are launched
 * round by round on their streams so that they overlap on the GPU.  results[i] receives flow i; wall_s
 * is the wall time of the whole batch.  Returns the first error status (all results are filled). */
tufrg_status tufrg_flow_batch(tufrg_model *const *models, int n, const tufrg_flow_opts *opts, tufrg_flow_result *results);

/* The flow of tufrg_flow driven step by step from the host, with checkpoints (the integration of Sec. 3.1 in the
 * flow variable ln T; the steps, the controller and the results are those of tufrg_flow).
 *
 * tufrg_flow_start: zeroes the state, evaluates k1 = f(y0) and captures one Dormand-Prince attempt, as tufrg_flow
 *   does before its first attempt; no attempt runs.  The model's work then runs on its private flow stream, ordered
 *   after the caller's stream, until tufrg_flow_end orders the caller's stream after it.  tufrg_flow and
 *   tufrg_flow_batch refuse a model with an open stepwise flow.
 * tufrg_flow_step: replays one attempt (nothing once the flow has stopped) and fills *info with the controller
 *   after it: T = exp(x) of the current accepted state, the next step h in ln T, the attempt's error norm, max |A|
 *   of the current state, the accepted-step and rejection counts, accepted (1 if this attempt was accepted) and
 *   status (0 running, 1 max |A| crossed the stop value, 2 reached T_end, 3 step limit, 4 non-finite, 5 step
 *   underflow).
 * tufrg_flow_amax_channels: h_amax[0], h_amax[1] = max |A_P|, max |A_C| over the projections of the last
 *   evaluated stage (after an accepted attempt: of the accepted state).
 * tufrg_flow_end: the tufrg_flow_result of what has run (wall_s from tufrg_flow_start or tufrg_flow_resume), the
 *   state to d_state_out (device, [2][Nq][M][M] complex FP64, may be NULL); closes the stepwise flow.  Returns the
 *   status tufrg_flow would return.
 * tufrg_flow_checkpoint_bytes: size of a checkpoint of this model (0 for NULL).
 * tufrg_flow_save: writes the open flow's checkpoint to the host buffer h_buf (caller-owned, at least
 *   tufrg_flow_checkpoint_bytes): a header (library version, model shape, channel mask, the products backend and
 *   loop launch shape in use), the device controller, the state y and k1 = f(y), FP64.
 * tufrg_flow_resume: opens a stepwise flow from a checkpoint of a model of the same shape and channel mask,
 *   restoring the controller, y and k1, and the checkpointed run's products backend and loop launch shape (they
 *   fix the summation order): the steps that follow are bit for bit those of the uninterrupted run.  opts gives
 *   the channel mask (the controller's scale range, tolerances and stop value come from the checkpoint).
 * Errors: TUFRG_EINVAL (NULL arguments, bad options, a second open flow, no open flow, a short buffer, a
 * checkpoint of another model, mask or library version), TUFRG_ENOTSUP (checkpoints of a model with a loop
 * surrogate), TUFRG_ENONFINITE (tufrg_flow_resume: a non-finite value in the checkpoint's state or derivative; the
 * model is left as it was), TUFRG_ETIMEOUT (a bounded device wait gave up), TUFRG_ECUDA, and tufrg_flow_end's flow
 * statuses. */
typedef struct {
    double T, h, err, amax;
    int n_steps, n_reject, accepted, status;
} tufrg_flow_step_info;
tufrg_status tufrg_flow_start(tufrg_model *m, const tufrg_flow_opts *opts);
tufrg_status tufrg_flow_step(tufrg_model *m, tufrg_flow_step_info *info);
tufrg_status tufrg_flow_amax_channels(tufrg_model *m, double *h_amax);
tufrg_status tufrg_flow_end(tufrg_model *m, void *d_state_out, tufrg_flow_result *result);
size_t tufrg_flow_checkpoint_bytes(const tufrg_model *m);
tufrg_status tufrg_flow_save(tufrg_model *m, void *h_buf, size_t bytes);
tufrg_status tufrg_flow_resume(tufrg_model *m, const tufrg_flow_opts *opts, const void *h_buf, size_t bytes);

/* ------------------------------------------------------------------------------------------
 * Learned loop surrogate (an addition with no counterpart in the paper).
 * A multilayer perceptron n_in -> [width, GELU] x depth -> n_out with BF16 weights, FP32
 * accumulation and FP32 master weights (Adam, mean-squared-error loss).  Training passes round the
 * activations to BF16; inference (tufrg_mlp_forward, the surrogate) keeps them in FP32.
 * Parameters are one flat FP32 vector: for each linear layer l, W_l [din][dout] row-major then
 * b_l [dout].  All device buffers are FP32, row-major [batch][features].
 * ------------------------------------------------------------------------------------------ */
typedef struct tufrg_mlp tufrg_mlp;
tufrg_status tufrg_mlp_create(int n_in, int width, int depth, int n_out, unsigned long long seed, void *cuda_stream,
                              tufrg_mlp **out);
void tufrg_mlp_free(tufrg_mlp *net);
const char *tufrg_mlp_last_error(const tufrg_mlp *net);
long long tufrg_mlp_num_params(const tufrg_mlp *net);
tufrg_status tufrg_mlp_get_params(tufrg_mlp *net, float *h_params);
tufrg_status tufrg_mlp_set_params(tufrg_mlp *net, const float *h_params);   /* also resets the Adam state */
tufrg_status tufrg_mlp_forward(tufrg_mlp *net, const float *d_X, int batch, float *d_Y);
/* gradient of the mean squared error mean((Y - T)^2) w.r.t. the flat parameters into d_grad */
tufrg_status tufrg_mlp_gradients(tufrg_mlp *net, const float *d_X, const float *d_T, int batch, float *d_grad, float *h_loss);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) on the batch; h_loss (may be NULL) receives the loss */
tufrg_status tufrg_mlp_train_step(tufrg_mlp *net, const float *d_X, const float *d_T, int batch, float lr, float *h_loss);

/* Attach a trained network as the loop surrogate of a split-precision two-band model (net = NULL
 * detaches).  Features per transfer momentum q = 2 pi (qx, qy)/Lq: sin(n qx), cos(n qx), sin(n qy),
 * cos(n qy) for n = 1..4, then (log T + 0.8)/3.1, (alpha - 0.2)/0.2, (t' + 0.15)/0.15, (mu + 0.9)/0.3 with
 * h_feature_params = {alpha, t', mu}.  Output j = ((ch*n_delta + d)*16 + ab)*2 + (0 re, 1 im) is
 * un-standardised as L = (y_j * h_std[j] + h_mean[j]) / T.  Every evaluation of the loops then checks
 * the surrogate against the direct k-sum at the n_check listed transfer momenta (relative Frobenius
 * norm over both channels) and falls back to the direct k-sum when the residual exceeds resid_tol.
 * A failed check switches the surrogate off (direct k-sum, network skipped) until it is re-armed:
 * tufrg_loops, tufrg_rhs, tufrg_rhs_host and every flow start re-arm it, so within a flow it serves
 * an unbroken first stretch.  All decisions are taken on the device.  The network must outlive its use
 * by the model. */
tufrg_status tufrg_set_surrogate(tufrg_model *m, tufrg_mlp *net, const float *h_mean, const float *h_std,
                                 const double *h_feature_params, double resid_tol, int n_check, const int *h_check_q);
/* Evaluations since the surrogate was attached that kept it, that fell back after a failed check, and
 * that skipped it because it was off (synchronises; any pointer may be NULL). */
tufrg_status tufrg_surrogate_stats(tufrg_model *m, long long *accepted, long long *rejected, long long *skipped);


/* Set (value != 0) or clear (value == 0) the model's device error flag, the flag a bounded device-side wait
 * (tensor-core pipeline barriers) raises when it gives up; an interface addition without a counterpart in the
 * paper.  While it is set, every call that reads it (tufrg_rhs_host, tufrg_rhs_host_batch, tufrg_flow,
 * tufrg_flow_batch) returns TUFRG_ETIMEOUT, so callers can test their handling of a time-out from the host without
 * making a device wait run out; clearing it makes the model usable again after a real time-out.  Synchronises
 * the model's stream.  Errors: TUFRG_EINVAL (NULL model), TUFRG_ECUDA. */
tufrg_status tufrg_set_device_error(tufrg_model *m, int value);

/* Optional CUDA-event timing on the model's stream (used by the benchmark).
 * tufrg_timing_begin resets the counters and starts recording; every later
 * kernel phase is bracketed by two events.  tufrg_timing_end synchronises the
 * stream, stops recording and returns:
 *   h_ms[i], i < n_ms: summed device milliseconds per phase, in the order
 *     0 Fermi tables, 1 loop k-sum kernels, 2 loop partial reduction,
 *     3 Fourier transform, 4 projections, 5 V.L.V products, 6 Runge-Kutta kernels, 7 the copy of the
 *     orbit representatives' products to the other momenta of their orbits (symmetric states, large M);
 *   *h_launches: kernels this library launched while recording;
 *   *h_loop_launches: launches of the loop k-sum kernel (phase 1) alone. */
tufrg_status tufrg_timing_begin(tufrg_model *m);
tufrg_status tufrg_timing_end(tufrg_model *m, double *h_ms, int n_ms, long long *h_launches, long long *h_loop_launches);

#ifdef __cplusplus
}
#endif
#endif /* TUFRG_H */
