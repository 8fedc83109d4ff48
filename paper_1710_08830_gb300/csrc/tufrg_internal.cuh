// Internal declarations shared by the translation units of libtufrg.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tufrg.h"

namespace tufrg {

// ------------------------------------------------------------------ small complex helpers
template <typename R> struct cpx;
template <> struct cpx<double> { using t = double2; };
template <> struct cpx<float> { using t = float2; };

__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }

// Fine-mesh Fermi table entry, one per (k, band): e = E - mu, g = df/dT, gp = dg/de.
struct FermiEntry {
    double e, g, gp;
};

// Split-precision copy used by the FP32 loop kernel.
struct FermiEntry32 {
    float e, g, gp, pad;
};
// With the momentum-shell regulator the same entries hold (e, f, h) at the fixed temperature T_reg:
// f = f(e), h = f (1 - f) / T_reg = -df/de (written once per model).

// Momentum-shell loop weight of one band pair (Eq. def_lmp): with (f, h) at the fixed temperature,
// F^- = (1 - f1 - f2) / (e1 + e2) (limit (h1 + h2) / 2), F^+ = (f1 - f2) / (e1 - e2) (limit
// -(h1 + h2) / 2), chi = e^2 / (e^2 + lam^2) and w = d/dlam [chi(e1) chi(e2)] F.
template <typename R> __device__ __forceinline__ R wdiv(R a, R b) { return a / b; }
template <> __device__ __forceinline__ float wdiv<float>(float a, float b) { return __fdividef(a, b); }
template <int WHICH, typename R>
__device__ __forceinline__ R shell_weight(R e1, R f1, R h1, R e2, R f2, R h2, R thr, R lam)
{
    R F;
    if (WHICH == 0) {
        const R s = e1 + e2;
        F = fabs(s) > thr ? wdiv<R>(R(1) - f1 - f2, s) : R(0.5) * (h1 + h2);
    } else {
        const R d = e1 - e2;
        F = fabs(d) > thr ? wdiv<R>(f1 - f2, d) : R(-0.5) * (h1 + h2);
    }
    const R l2 = lam * lam, a1 = e1 * e1, a2 = e2 * e2;
    const R q1 = a1 + l2, q2 = a2 + l2;
    // d/dlam [a1 a2 / (q1 q2)] = -2 lam a1 a2 (q1 + q2) / (q1 q2)^2
    const R p = q1 * q2;
    return wdiv<R>(R(-2) * lam * a1 * a2 * (q1 + q2), p * p) * F;
}

// Loop weight of one band pair: d/dT F^- = -(g1 + g2) / (e1 + e2) (WHICH = 0) or d/dT F^+ = (g1 - g2) / (e1 - e2)
// (WHICH = 1) from the Fermi entries (e, g, g'), with the limit -+(g'1 + g'2) / 2 below |e1 -+ e2| = thr; with
// lam > 0 the momentum-shell weight above, the entries then holding (e, f, h).
template <int WHICH, typename R>
__device__ __forceinline__ R gen_pair_weight(R e1, R g1, R gp1, R e2, R g2, R gp2, R thr, R lam)
{
    if (lam > R(0)) return shell_weight<WHICH, R>(e1, g1, gp1, e2, g2, gp2, thr, lam);   // (g, gp) = (f, h)
    if (WHICH == 0) {
        const R s = e1 + e2;
        return fabs(s) > thr ? -(g1 + g2) / s : R(-0.5) * (gp1 + gp2);
    } else {
        const R d = e1 - e2;
        return fabs(d) > thr ? (g1 - g2) / d : R(0.5) * (gp1 + gp2);
    }
}

// Everything the projection kernel needs about one gather term.
// kind: 0 = P<-C, 1 = P<-D, 2 = C<-P, 3 = C<-D.
struct GatherTerm {
    int cls;   // row of the Fourier-transformed source (bond class of R'' or -R')
    int i1, i2;
    int ph;    // column of the phase table e^{i q.R}
    int kind;
};

// Device-resident state of one adaptive flow (Dormand-Prince 5(4) in x = ln T).
struct FlowDev {
    double x, h, xend, x_prev;
    double amax_prev, amax, Tc, err;
    double atol, rtol, stop;
    int n_steps, n_reject, tries, max_tries;
    int status;       // 0 running, 1 crossed the stop value, 2 reached T_end, 3 step limit, 4 non-finite, 5 step underflow
    int accepted;     // 1 if the last attempt was accepted
};

// One element of the loop symmetry group: Lc(q')[d'][a'][b'] = i^(qt[ch][a'] - qt[ch][b']) *
// (conj ? conj(L) : L) with L = Lc(q)[d][src[ch][a']][src[ch][b']], q' = G_q q, Delta_d' = G Delta_d
// (orbital-pair indices a < N_s^2 <= 36; every phase is a power of i).
constexpr int SYM_MAXNS2 = 36;
struct SymElem {
    int conj;
    int src[2][SYM_MAXNS2];
    int qt[2][SYM_MAXNS2];
};

// (hi, lo) words of the exact double of a float, formed on the integer pipe only (this GPU's FP64 pipe,
// which also executes conversions, is slow; a branch to a plain conversion gets if-converted into an
// unconditional one): normal, zero, subnormal (normalised with clz), inf and nan.
static __device__ __noinline__ uint2 widen_general(float f)
{
    const unsigned u = __float_as_uint(f), sign = u & 0x80000000u, e = (u >> 23) & 0xffu, man = u & 0x7fffffu;
    if (e == 0xffu) return make_uint2(sign | 0x7ff00000u | (man >> 3), man << 29);
    if (e != 0u) return make_uint2(sign | ((e + 896u) << 20) | (man >> 3), man << 29);
    if (man == 0u) return make_uint2(sign, 0u);
    const int p = 31 - __clz((int)man);   // leading bit of the subnormal mantissa, value = man 2^-149
    const unsigned long long fr = (unsigned long long)(man & ((1u << p) - 1u)) << (52 - p);
    return make_uint2(sign | ((unsigned)(p - 149 + 1023) << 20) | (unsigned)(fr >> 32), (unsigned)fr);
}
// The same with a fast path for normal values and zeros (the exponent rebiased, the significand moved
// down 3 bits into the high word, its low 3 bits to the top of the low word).
__device__ __forceinline__ uint2 widen_bits(float f)
{
    const unsigned u = __float_as_uint(f), a = u & 0x7fffffffu, sign = u & 0x80000000u;
    if (a - 0x00800000u < 0x7f000000u) return make_uint2(sign | ((a >> 3) + (896u << 20)), a << 29);
    if (a == 0u) return make_uint2(sign, 0u);
    return widen_general(f);
}

__device__ __forceinline__ double widen_f(float f)
{
    const uint2 w = widen_bits(f);
    return __hiloint2double((int)w.x, (int)w.y);
}

// FP64 -> FP32 rounding to nearest, ties to even (IEEE 754 convertFormat), on the integer pipe for the
// same reason, without branches (a branch per value stalls the loads that feed it): the 53-bit
// significand (hidden bit included) is shifted right by 29 places, more for a subnormal or zero result,
// and rounded on the discarded bits; a carry out of the significand increments the exponent field,
// which also turns the largest finite values into infinity where they round up.  Results beyond the
// FP32 range, infinities and NaNs (quiet, top payload bits kept) are selected at the end.
static __device__ __noinline__ float narrow_general(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned long long man = b & 0xfffffffffffffull;
    const int E0 = e - 896;                                     // biased FP32 exponent of a normal result
    const int shift = min(29 + max(0, 1 - E0), 63);
    const unsigned long long sig = man | (e ? (1ull << 52) : 0ull);
    const unsigned long long kept = sig >> shift, rem = sig & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
    const unsigned r = (unsigned)kept + ((rem > half || (rem == half && (kept & 1ull))) ? 1u : 0u);
    // normal: (E - 1) << 23 plus the significand with its hidden bit; subnormal: the significand alone
    unsigned bits = (E0 > 0 ? (unsigned)(E0 - 1) << 23 : 0u) + r;
    bits = E0 >= 255 ? 0x7f800000u : bits;
    bits = e == 0x7ff ? 0x7f800000u | (man ? 0x400000u | (unsigned)(man >> 29) : 0u) : bits;
    return __uint_as_float(sign | bits);
}

// The same rounding with a 32-bit fast path for zeros and normal FP32 results (biased FP64 exponent in
// [897, 1150]): the FP32 exponent and significand are the FP64 fields above the 29 discarded bits,
// rebiased; the rest takes the general path.
__device__ __forceinline__ float narrow_f(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b, habs = hi & 0x7fffffffu;
    if (habs - (897u << 20) < (254u << 20)) {
        const unsigned f = __funnelshift_l(lo, habs - (896u << 20), 3);   // rebiased exponent | top 23 bits
        const unsigned rem = lo & 0x1fffffffu;
        const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
        return __uint_as_float((hi & 0x80000000u) | (f + up));
    }
    if ((habs | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return narrow_general(x);
}

// 16-byte asynchronous copy global -> shared (L2 only), and the waits on this thread's own copy groups
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

struct LoopPlan {
    int kx_per_cta;     // threads (columns) per CTA
    int ky_chunks;      // number of ky ranges per column
    int n_partials;     // partial sums per transfer momentum
};

}  // namespace tufrg

struct tufrg_mlp;

struct tufrg_model {
    // ---- descriptor copy
    int ns = 0, nhop = 0, nff = 0, Lq = 0, nc = 0, Lf = 0, Nq = 0, Nk = 0, M = 0, precision = 0;
    int regulator = 0;      // TUFRG_REG_TEMPERATURE / TUFRG_REG_MOMENTUM_SHELL
    double T_reg = 0.0;     // momentum shell: temperature of the Fermi functions
    std::vector<int> hopR, ffR;
    std::vector<double> hopt, V0;
    double mu = 0.0;
    cudaStream_t stream = nullptr;
    std::string err;
    int sm_count = 0;

    // ---- bond bookkeeping (host)
    std::vector<int> deltas;        // [nd][2] sorted (dx, dy)
    int nd = 0;
    std::vector<int> dxs, dys;      // distinct dx / dy values (sorted)
    std::vector<int> dslot;         // [nd] see d_dslot
    std::vector<int> dpartner;      // [nd] index of -delta
    std::vector<int> dij;           // [nff][nff] -> delta index of R1 - R2
    std::vector<int> cls;           // [ncls][2] bond classes mod Lq used by projections
    int ncls = 0;
    std::vector<int> phv;           // [nph][2] phase vectors mod Lq
    int nph = 0;
    std::vector<int> gofs[2];       // CSR offsets per output channel, [nff*nff + 1]
    std::vector<tufrg::GatherTerm> gterms[2];
    std::vector<int> gtab_export[2];  // 9 ints per term, for tufrg_gather_table

    // ---- device memory (owned)
    double *d_E = nullptr;          // [Nk][ns]
    double2 *d_U = nullptr;         // [Nk][ns][ns]
    float2 *d_U32 = nullptr;        // [Nk][ns][ns] (split path)
    tufrg::FermiEntry *d_ft = nullptr;      // [Nk][ns]
    tufrg::FermiEntry32 *d_ft32 = nullptr;  // [Nk][ns]
    int *d_dslot = nullptr;         // [nd] partial slot (dxi * ndyh + dyi) of the half-plane partner
    int *d_deltas = nullptr;        // [nd][2]
    int *d_dpartner = nullptr;      // [nd] index of -delta
    int *d_hopR = nullptr;          // [nhop][2]
    double2 *d_hopt = nullptr;      // [nhop][ns][ns]
    double *d_scal = nullptr;       // device scalars: [0] temperature of the current evaluation, [1] product scale
    int *d_dij = nullptr;           // [nff][nff]
    int *d_gofs[2] = {nullptr, nullptr};
    tufrg::GatherTerm *d_gterms[2] = {nullptr, nullptr};
    // loop symmetries (TUFRG_SYMMETRY_AUTO): the k-sums run for one representative momentum per orbit
    // of the symmetry group and the reduction writes every orbit member from it
    bool sym = false;
    int n_loop_q = 0;               // transfer momenta summed directly (Nq without symmetry)
    int n_sym_elem = 0;             // group elements (identity included)
    int *d_loop_list = nullptr;     // [n_loop_q] orbit representatives
    int2 *d_qmap = nullptr;         // [Nq] (list position of the orbit representative, group element)
    tufrg::SymElem *d_sym_elem = nullptr;   // [n_sym_elem]
    int *d_sym_dinv = nullptr;      // [n_sym_elem][nd] source d of target d' (Delta_d' = G Delta_d)
    // symmetric states (flows from X = 0 with a symmetric bare vertex): X(G q) = W X(q) W^dagger with W the
    // element's bond permutation times its orbital-pair map, so projections and products run for the orbit
    // representatives only and dX/dT of the other momenta is gathered from them
    bool sym_state = false;
    double sym_tune_ms[2] = {-1.0, -1.0};   // projections + products at every momentum / representatives + gather
    int *d_sym_srow = nullptr;      // [n_sym_elem][2][M] source index of every target row / column
    int *d_sym_qrow = nullptr;      // [n_sym_elem][2][M] quarter turns of every target row / column
    int *d_sym_sinv = nullptr;      // [n_sym_elem][2][M] target index of every source row (srow inverted), or null
    int *d_orb_ofs = nullptr;       // [n_loop_q + 1] orbit of each representative: momenta orb_q[ofs[p] .. ofs[p+1])
    int *d_orb_q = nullptr;         // [Nq]
    int *d_sym_emap = nullptr;      // [n_sym_elem][2][M^2] source entry << 3 | quarter turns << 1 | conj (small M)
    int *d_orb_lexp = nullptr;      // [M^2] compact-loop index of every expanded loop-matrix entry (small M)
    void *d_band_tc = nullptr;      // [2][Nq][n_delta][16] compact band-basis transformation matrices
    int *d_eofs[2] = {nullptr, nullptr};       // per output channel: CSR offsets per matrix entry, [M*M + 1]
    int2 *d_eterms[2] = {nullptr, nullptr};    // per entry terms: (flat index into the Fourier transforms,
                                               //  high bit = minus sign; phase-table column)
    double2 *d_v0d[2] = {nullptr, nullptr};    // [M*M] bare vertex V0 at the onsite bond pair, 0 elsewhere
    float2 *d_X32 = nullptr;        // [2][Nq][M][M] FP32 copy of the state being evaluated (split path)
    float2 *d_lph32 = nullptr;      // [Lf] e^{-2 pi i n / Lf} for the split loop kernel
    float2 *d_clsph32 = nullptr;    // [Nq][ncls] e^{i u.R''} (split-path Fourier transform)
    float2 *d_v0d32[2] = {nullptr, nullptr};   // FP32 copies of d_v0d (split path)
    double2 *d_ph = nullptr;        // [Nq][nph] phase table e^{i q.R}
    double2 *d_clsph = nullptr;     // [Nq][ncls] e^{i q.R''} for the Fourier transform
    double2 *d_V0 = nullptr;        // [ns^4]
    double2 *d_Lc = nullptr;        // [2][Nq][nd][ns^4] loops (FP64 view)
    float2 *d_Lc32 = nullptr;       // [2][Nq][nd][ns^4] loops (split path)
    void *d_part = nullptr;         // loop partial sums (scratch)
    size_t part_bytes = 0;
    double2 *d_Xr = nullptr;        // [2][ncls][M][M] Fourier transforms
    double2 *d_A = nullptr;         // [2][Nq][M][M] projected vertex
    float2 *d_A32 = nullptr;        // [2][Nq][M][M] (split path)
    double2 *d_T = nullptr;         // [Nq][M][M] GEMM intermediate (large M); split: [2][Nq][M][M] FP32 complex
    float4 *d_rec = nullptr;        // [Nk][4] split-path loop records (projectors + Fermi data)
    float2 *d_Xr32 = nullptr;       // [2][ncls][M][M] Fourier transforms (split path)
    float2 *d_ph32 = nullptr;       // [Nq][nph] phase table (split path)
    void *d_dftpart = nullptr;      // Fourier-transform scratch: partial sums, or Z(u_x, R_y) of the separable form
    int dft_nsplit = 1;             // transfer-mesh slices of the Fourier transform
    // separable Fourier transform: distinct R_y / R_x of the classes, warps per CTA of its column pass (the most
    // classes with one R_y; 0 = not used), int tables (class id by R_y group, R_x index, R_y group offsets) and
    // phases [Lq][n_Ry], [Lq][n_Rx]; its row pass keeps Z(u_x, R_y) in d_dftpart
    int dft_nry = 0, dft_nrx = 0, dft_warps = 0;
    int *d_dft_tabs = nullptr;
    double2 *d_dft_phy = nullptr, *d_dft_phx = nullptr;
    float2 *d_dft_phy32 = nullptr, *d_dft_phx32 = nullptr;
    int max_terms = 0;              // largest gather-term list of one (R, R') pair
    unsigned long long *d_amax = nullptr;   // [4] reductions (max|A|, argmax, err)
    int *d_err = nullptr;           // device-side error flag (bounded waits)
    int products = TUFRG_PRODUCTS_SIMT;     // backend of the split-path products
    double tune_ms[2] = {-1.0, -1.0};       // autotuner timings (tensor cores, CUDA cores)
    int tc_ntiles = 0;                       // tensor-core products: column tiles per matrix (0: the fewest)
    std::vector<double> tc_tile_ms;         // the products autotuner's timings of the column-tile candidates
    double *d_red = nullptr;        // density reduction scratch
    // flow work buffers
    double2 *d_y = nullptr, *d_yt = nullptr, *d_yn = nullptr, *d_k[7] = {};
    double2 *d_state_in = nullptr, *d_state_out = nullptr;   // host-buffer entry points
    // pipelined host-buffer evaluations: two device buffers per direction, one stream per copy direction,
    // and per buffer the events "input copied", "evaluated", "output copied"
    double2 *d_bin[2] = {nullptr, nullptr}, *d_bout[2] = {nullptr, nullptr};
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    tufrg::FlowDev *d_flow = nullptr;        // device controller state
    tufrg::FlowDev *h_flow = nullptr;        // pinned host mirror
    cudaGraphExec_t step_graph = nullptr;    // one captured Dormand-Prince attempt
    cudaStream_t flow_stream = nullptr;      // private capturable stream of the flow (joined to `stream` by events)
    // second stream of a right-hand side: the Fourier transform and projections (they read the state only) run
    // there while the loop k-sum (it reads the temperature only) runs on `stream`; joined before the products
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t aux_ev[2] = {nullptr, nullptr};
    cudaEvent_t flow_ev = nullptr;
    // tufrg_rhs replays captured graphs of its launches, one per (input, output, mask) used more than once (the
    // four most recently used triples kept; exec is null after the first use)
    struct RhsGraph {
        const void *in;
        void *out;
        int mask;
        cudaGraphExec_t exec;
        long long launches, loop_launches;   // kernels the graph holds (the launch counters advance by these)
        unsigned long long used;
    };
    std::vector<RhsGraph> rhs_graphs;
    unsigned long long rhs_graph_clock = 0;
    bool rhs_graph_off = false;              // a capture failed once: launch directly from then on
    cudaStream_t rhs_stream = nullptr;       // private stream of the graphs when the model's stream is the legacy one
    cudaEvent_t rhs_ev[2] = {nullptr, nullptr};
    // a flow driven step by step from the host (tufrg_flow_start .. tufrg_flow_end)
    bool flow_open = false;
    cudaStream_t flow_user = nullptr;        // the caller's stream, rejoined at the end
    int flow_mask = 0;
    double flow_t0 = 0.0;                    // host clock at the start (seconds)
    unsigned long long *d_amax_ch = nullptr; // [2] max |A| per channel (bit patterns of non-negative doubles)
    int step_graph_mask = 0;

    tufrg::LoopPlan plan{};
    std::vector<tufrg::LoopPlan> plan_cand;   // timed launch shapes of the loop k-sum (two-band split path)
    std::vector<double> plan_ms;              // their measured times (ms per launch), same order
    int gen_chunks = 1;             // multi-orbital loop kernel: kx ranges (CTAs, accumulator slots) per momentum
    int basis = TUFRG_BASIS_ORBITAL;   // single-particle basis of the flow
    std::vector<double> ffW;        // [nff][nff] irrep form factors over the bonds (empty: set not C4v-closed)
    std::vector<int> ff_labels;     // [nff][3] (shell, irrep A1 A2 B1 B2 E, partner)
    double *d_ffW = nullptr;
    double2 *d_v0q = nullptr;       // band basis: [2][Nq][M][M] projected bare vertex per momentum (FP64)
    float2 *d_v0q32 = nullptr;      // its FP32 copy (split path)
    int *d_shard_q = nullptr;       // [Nq] momenta of a shard (sharded right-hand side)
    double2 *d_shard_out = nullptr; // [2][Nq][M][M] products of a shard's momenta before they are gathered
    bool loops_tc = false;          // multi-orbital loop k-sum on the tensor cores (k_loops_tc.cu)
    float2 *d_loop_w = nullptr;     // its column sums [groups][Lf][108][108]

    // ---- learned loop surrogate (optional)
    tufrg_mlp *sur = nullptr;       // network (not owned)
    double sur_tol = 1e-3;          // relative Frobenius residual accepted at the check momenta
    double sur_params[3] = {0, 0, 0};   // alpha, t', mu features of this model
    int n_check = 0;
    int *d_check_q = nullptr;       // [n_check] transfer momenta of the residual check
    float *d_sur_X = nullptr;       // [Nq][20] features
    float *d_sur_Y = nullptr;       // [Nq][n_out] network output (standardised)
    float *d_sur_mean = nullptr, *d_sur_std = nullptr;   // [n_out]
    float2 *d_chk_part = nullptr;   // partial sums of the check momenta
    double2 *d_chk = nullptr;       // [2][n_check][nd][16] direct loops at the check momenta
    int *d_sur_flag = nullptr;      // [0] 1: surrogate accepted for this evaluation (direct k-sum skipped)
                                    // [1] 1: a check failed since the last re-arm; surrogate off until then
    unsigned long long *d_sur_count = nullptr;   // [3] accepted, rejected, skipped

    // ---- optional event timing (phases as listed in tufrg.h)
    bool timing = false;
    long long launches = 0, loop_launches = 0;
    struct TimerRec { int phase; cudaEvent_t a, b; };
    std::vector<TimerRec> trec;
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
};

namespace tufrg {

// ------------------------------------------------------------------ launchers (k_*.cu)
cudaError_t launch_bands(tufrg_model *m);
cudaError_t launch_density(tufrg_model *m, double mu, double T, double *h_out);
cudaError_t launch_fermi(tufrg_model *m);
cudaError_t launch_set_scalars(tufrg_model *m, double T, double scale);
// reps_only (with loop symmetries): the FP32 loops of the orbit representatives only, at their own
// momenta, and no FP64 copy on the split path (what the symmetric-state products read)
cudaError_t launch_loops(tufrg_model *m, int channel_mask, bool reps_only = false);
// The split path reads the FP32 copy of the state (d_state32), the plain path the FP64 state.
// whether the separable transform applies: *warps = warps per CTA of its column pass, 0 if it does not
void dft_sep_plan(const tufrg_model *m, int *warps);
cudaError_t launch_dft(tufrg_model *m, const double2 *d_state, const float2 *d_state32, int channel_mask);
// qlist (nlist entries): only these transfer momenta (the orbit representatives of a symmetric state)
cudaError_t launch_project(tufrg_model *m, const double2 *d_state, const float2 *d_state32, int channel_mask,
                           double2 *d_A, const int *qlist = nullptr, int nlist = 0);
cudaError_t launch_to_f32(tufrg_model *m, const double2 *d_state, float2 *d_out, size_t n);
cudaError_t launch_widen_f64(const float *d_in, double *d_out, size_t n, cudaStream_t stream);
cudaError_t launch_round_f32(const double *d_in, float *d_out, size_t n, cudaStream_t stream);
// qlist (nlist entries): only these transfer momenta
cudaError_t launch_vlv(tufrg_model *m, const double2 *d_A, int channel_mask, double2 *d_out, const int *qlist = nullptr,
                       int nlist = 0);
cudaError_t launch_rk_combine(tufrg_model *m, double2 *out, float2 *out32, const double2 *y, const FlowDev *fs,
                              const double *a, double2 *const *k, int nk, size_t n);
cudaError_t launch_rk_error(tufrg_model *m, const double2 *y, const double2 *yn, const FlowDev *fs, const double *e,
                            double2 *const *k, int nk, size_t n);
cudaError_t launch_stage_scalars(tufrg_model *m, const FlowDev *fs, double cj);
cudaError_t launch_flow_init(tufrg_model *m, FlowDev *fs);
cudaError_t launch_flow_decide(tufrg_model *m, FlowDev *fs);
cudaError_t launch_flow_commit(tufrg_model *m, const FlowDev *fs, double2 *y, const double2 *yn, double2 *k0,
                               const double2 *k6, size_t n);
cudaError_t launch_amax_channels(tufrg_model *m, bool reps_only);
cudaError_t launch_amax_locate(tufrg_model *m, size_t n, bool reps_only);   // on the last projection (d_A or d_A32)
LoopPlan plan_loops(const tufrg_model *m);
void drop_rhs_graphs(tufrg_model *m);
// the launch shapes the two-band split loop kernel's autotuner times (ky ranges per column)
std::vector<LoopPlan> loop_plan_candidates(const tufrg_model *m);
int plan_gen_chunks(const tufrg_model *m);   // kx ranges per momentum of the multi-orbital loop kernel
size_t gen_red_offset(const tufrg_model *m);   // byte offset of the representatives' range sums in d_part
size_t gen_part_bytes(const tufrg_model *m);   // loop scratch of the multi-orbital kernel
int dft_plan_nsplit(const tufrg_model *m);
bool loops2_supported(const tufrg_model *m);
int loops2_blocks_per_sm(const tufrg_model *m);
bool loops_gen_supported(const tufrg_model *m);
cudaError_t launch_loops_gen(tufrg_model *m, int channel_mask, bool reps_only);
// sharded right-hand side (k_shard.cu): a shard's part of the Fourier transform, the gather of its rows, and the
// loops at a list of momenta
cudaError_t launch_shard_dft(tufrg_model *m, const double2 *d_state_local, int n, const int *d_q, int mask, double2 *d_xr);
cudaError_t launch_shard_gather(tufrg_model *m, const double2 *d_full, int n, const int *d_q, double2 *d_out);
cudaError_t launch_loops_list(tufrg_model *m, int mask, const int *d_list, int n);
// projections of the listed momenta whose state rows are stored in list order, [2][nlist][M][M]
cudaError_t launch_project_local(tufrg_model *m, const double2 *d_state_local, const float2 *d_state32_local,
                                 int channel_mask, double2 *d_A, const int *qlist, int nlist);
// form factors of the irreducible representations of C4v (k_irrep.cu)
bool build_irrep_basis(tufrg_model *m);
cudaError_t launch_irrep_basis(tufrg_model *m, const double2 *d_state, int inverse, double2 *d_out);
bool loops_tc_supported(const tufrg_model *m);
size_t loops_tc_w_bytes(const tufrg_model *m);
cudaError_t launch_loops_tc(tufrg_model *m, int ch, float2 *acc);
cudaError_t launch_vlv_large(tufrg_model *m, const double2 *d_A, int channel_mask, double2 *d_out, const int *qlist,
                             int nlist);
cudaError_t launch_sym_scatter(tufrg_model *m, double2 *d_out);
// symmetric states: products at the orbit representatives and dX/dT of every momentum (the fused orbit
// kernel where its tables exist, else the representatives' products plus the scatter)
cudaError_t launch_products_sym(tufrg_model *m, int channel_mask, double2 *d_out);
// band-basis exchange propagators of a two-band model's state (Sec. 3.4)
bool band_basis_supported(const tufrg_model *m);
// band-basis flow: the projected bare vertex per momentum from the model's eigenvectors, then unit eigenvectors
cudaError_t setup_band_flow(tufrg_model *m);
cudaError_t launch_band_basis(tufrg_model *m, const double2 *d_state, double2 *d_out);
bool orbit_products_supported(const tufrg_model *m);
int orbit_max_size();   // largest orbit the fused orbit kernel takes   // symmetric states: non-representative momenta
bool tc_supported(const tufrg_model *m);
std::vector<int> tc_tile_candidates(const tufrg_model *m);
int tc_tile_width(const tufrg_model *m);
cudaError_t launch_vlv_tc(tufrg_model *m, int channel_mask, double2 *d_out, const int *qlist, int nlist);
cudaError_t launch_loop_records(tufrg_model *m);          // per evaluation: Fermi data at d_scal[0]
cudaError_t launch_loop_records_static(tufrg_model *m);   // once per model: projectors and e = E - mu
cudaError_t launch_loop_records_shell(tufrg_model *m);    // once per model (momentum shell): f, h at T_reg
cudaError_t launch_fermi_shell(tufrg_model *m);           // once per model (momentum shell): (e, f, h) tables
cudaError_t launch_loops2(tufrg_model *m, int ch);
cudaError_t launch_loops2_ex(tufrg_model *m, int ch, const int *s_list, int n_list, float2 *part, const int *skip);
cudaError_t launch_surrogate(tufrg_model *m, int channel_mask);
cudaError_t mlp_forward_on(tufrg_mlp *n, cudaStream_t s, const float *X, int batch, float *Y, const int *skip);
// the network's GEMMs on the tensor cores (k_mlp_tc.cu); TA = __nv_bfloat16 (training) or float (inference)
size_t mlp_tc_scratch_bytes(int M, int N, int K);
template <typename TA>
cudaError_t mlp_gemm_tc(cudaStream_t s, const TA *A, int lda, int ta, const struct __nv_bfloat16 *B, int ldb, int tb,
                        float *C, int ldc, int M, int N, int K, const float *bias, const int *skip, void *ws, int *err);
cudaError_t surrogate_rearm(tufrg_model *m);
void mlp_dims(const tufrg_mlp *n, int *n_in, int *n_out);

enum Phase { PH_FERMI = 0, PH_LOOPS = 1, PH_LOOPRED = 2, PH_DFT = 3, PH_PROJ = 4, PH_VLV = 5, PH_RK = 6, PH_SCATTER = 7, PH_N = 8 };

// Brackets one kernel phase with events when timing is on; counts launches always.
struct PhaseScope {
    tufrg_model *m;
    int idx = -1;
    PhaseScope(tufrg_model *mm, int phase, int n_launch = 1);
    ~PhaseScope();
};

}  // namespace tufrg

#define TUFRG_CUDA_TRY(expr)                                  \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return _e;                     \
    } while (0)
