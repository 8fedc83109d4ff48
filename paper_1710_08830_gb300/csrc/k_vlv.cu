// dX/dT(q) = c_X A_X(q) L_X(q) A_X(q): Sec. 4.2 Eq. RGE_spin (c_P = 1) and the orbital
// form of Eq. rge_Dmat (c_C = 2).  The M x M loop matrix is never stored: it is
// expanded from the compact loops, L[(R1,a),(R2,b)] = Lc[d(R1-R2)][a][b].
//
// Small M (<= 64): one CTA per (q, channel) holds A, L and the intermediate
// T = A L in shared memory and writes c * T A.  For two-band bond sets
// (M = 4 N_ff) every thread owns a 4 x 4 tile of each product (16 complex FMAs
// per four conflict-free 16-byte shared loads), and two M x M buffers serve
// both products so that one wave of CTAs covers all transfer momenta.  FP64 for the plain path;
// FP32 arithmetic on the FP32 copies for the split path, whose FP64 output is
// widened exactly on the integer pipe (this GPU's FP64 pipe would bound it).
#include <algorithm>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

template <typename C2> __device__ __forceinline__ void cfma(C2 &acc, C2 a, C2 b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// one FP64 complex output (little-endian double2 = lo, hi, lo, hi words)
__device__ __forceinline__ void store_c(double2 *o, float2 v, float sc)
{
    const uint2 re = widen_bits(sc * v.x), im = widen_bits(sc * v.y);
    *reinterpret_cast<uint4 *>(o) = make_uint4(re.y, re.x, im.y, im.x);
}
__device__ __forceinline__ void store_c(double2 *o, double2 v, double sc) { *o = make_double2(sc * v.x, sc * v.y); }

// two consecutive complex values from 16-byte aligned shared memory
__device__ __forceinline__ void ld2(const float2 *p, float2 &a, float2 &b)
{
    const float4 u = *reinterpret_cast<const float4 *>(p);
    a = make_float2(u.x, u.y);
    b = make_float2(u.z, u.w);
}
__device__ __forceinline__ void ld2(const double2 *p, double2 &a, double2 &b)
{
    a = p[0];
    b = p[1];
}

// acc[i][j] += sum_k X[k][row_i] Y[k][col_j] for the 4 x 4 tile with rows {r, r+1, r+h, r+h+1} and
// columns {c, c+1, c+h, c+h+1} (h = M/2); X is stored transposed (k-major), so both operands are read
// as pairs of 16-byte chunks that consecutive lanes take from consecutive addresses.
template <typename C2>
__device__ __forceinline__ void tile44(const C2 *Xt, const C2 *Y, int M, int r, int c, C2 acc[4][4])
{
    const int h = M / 2;
    for (int k = 0; k < M; k++) {
        C2 a[4], b[4];
        ld2(Xt + k * M + r, a[0], a[1]);
        ld2(Xt + k * M + h + r, a[2], a[3]);
        ld2(Y + k * M + c, b[0], b[1]);
        ld2(Y + k * M + h + c, b[2], b[3]);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) cfma(acc[i][j], a[i], b[j]);
    }
}

// The same contraction for the 2 x 2 tile with rows {r, r+1} and columns {c, c+1} (r, c even): every
// output element sees the same sequence of complex FMAs over k as in tile44.
template <typename C2>
__device__ __forceinline__ void tile22(const C2 *Xt, const C2 *Y, int M, int r, int c, C2 acc[2][2])
{
    for (int k = 0; k < M; k++) {
        C2 a0, a1, b0, b1;
        ld2(Xt + k * M + r, a0, a1);
        ld2(Y + k * M + c, b0, b1);
        cfma(acc[0][0], a0, b0);
        cfma(acc[0][1], a0, b1);
        cfma(acc[1][0], a1, b0);
        cfma(acc[1][1], a1, b1);
    }
}

// an FP32 value widened exactly to FP64 on the integer pipe
__device__ __forceinline__ void store_w(double2 *o, float2 v)
{
    const uint2 re = widen_bits(v.x), im = widen_bits(v.y);
    *reinterpret_cast<uint4 *>(o) = make_uint4(re.y, re.x, im.y, im.x);
}

// Symmetric states, two-band bond sets (M = 4 N_ff <= 64), split path.  One CTA per (orbit
// representative q, channel) forms c A L A at q with one 2 x 2 output tile per thread ((M/2)^2 threads;
// per element the same FP32 arithmetic as vlv_tiled_kernel) and writes dX/dT of every momentum q' of the
// orbit from the result R held in shared memory:
//   out[q'][t] = i^turns (conj ? conj(R[src]) : R[src]),
// e the element that maps q to q' (the representative itself is written as is).  The index map holds the
// composed transform, emap[e][ch][t] = src << 3 | swap << 2 | negate_re << 1 | negate_im: with
// w = R[src], out = (+-(swap ? w.y : w.x), +-(swap ? w.x : w.y)).  Every thread owns at
// most ORB_UNITS entries of each matrix pass; the loads of a pass are issued before their uses, the
// orbit's momenta and elements sit in shared memory, and the stores are coalesced.  lexp[t] is the
// compact-loop index of expanded entry t, L[(R1,a),(R2,b)] = Lc[d(R1-R2)][a][b].
constexpr int ORB_MAX = 32;     // orbit size bound (the square lattice's 8 operations, times time reversal)
constexpr int ORB_UNITS = 4;    // entries per thread per pass (blockDim >= M^2 / 4)

__global__ void __launch_bounds__(1024) vlv_orbit_kernel(const float2 *__restrict__ A, const float2 *__restrict__ Lc,
                                                         const int *__restrict__ lexp, int Nq, int M, int nd,
                                                         int chmask, const double *scal, const int *list,
                                                         const int *orb_ofs, const int *orb_q, const int2 *qmap,
                                                         const int *__restrict__ emap, double2 *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *s0 = reinterpret_cast<float2 *>(smem_raw);   // A^T, then A, then the result R
    float2 *s1 = s0 + M * M;                              // L, then T^T
    __shared__ int s_q2[ORB_MAX], s_e[ORB_MAX];           // the orbit's momenta and elements (-1: q itself)
    const int p = blockIdx.x, ch = blockIdx.y, q = list[p];
    const int M2 = M * M, nt = M / 2, B = blockDim.x;
    const int m0 = orb_ofs[p], nmem = orb_ofs[p + 1] - m0;
    if ((int)threadIdx.x < nmem) {
        const int q2 = orb_q[m0 + threadIdx.x];
        s_q2[threadIdx.x] = q2;
        s_e[threadIdx.x] = q2 == q ? -1 : qmap[q2].y;
    }
    const bool on = (chmask >> ch) & 1;
    const float2 *a = A + ((size_t)ch * Nq + q) * M2;
    const float2 *lc = Lc + ((size_t)ch * Nq + q) * nd * 16;
    float2 av[ORB_UNITS];
    if (on) {
        // A^T and the expanded loop matrix; (r, c) of entry i advance incrementally (B = dr M + dc, dc < M)
        const int dr = B / M, dc = B - dr * M;
        int li[ORB_UNITS], rr[ORB_UNITS], cc[ORB_UNITS];
        int r = threadIdx.x / M, c = threadIdx.x - r * M;
#pragma unroll
        for (int u = 0; u < ORB_UNITS; u++) {
            const int i = threadIdx.x + u * B;
            av[u] = i < M2 ? a[i] : make_float2(0.f, 0.f);
            li[u] = i < M2 ? lexp[i] : 0;
            rr[u] = r;
            cc[u] = c;
            r += dr;
            c += dc;
            if (c >= M) {
                c -= M;
                r++;
            }
        }
        float2 lv[ORB_UNITS];
#pragma unroll
        for (int u = 0; u < ORB_UNITS; u++) lv[u] = threadIdx.x + u * B < M2 ? lc[li[u]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < ORB_UNITS; u++) {
            const int i = threadIdx.x + u * B;
            if (i < M2) {
                s0[cc[u] * M + rr[u]] = av[u];
                s1[i] = lv[u];
            }
        }
    }
    __syncthreads();
    if (on) {
        const bool active = (int)threadIdx.x < nt * nt;
        const int ti = threadIdx.x / nt, tj = threadIdx.x - ti * nt;
        const int r = 2 * ti, c = 2 * tj;
        float2 acc[2][2];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) acc[i][j] = make_float2(0.f, 0.f);
        if (active) tile22(s1, s0, M, r, c, acc);   // T^T = L^T A^T
        __syncthreads();
        if (active) {
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    s1[(r + i) * M + c + j] = acc[i][j];
                    acc[i][j] = make_float2(0.f, 0.f);
                }
        }
#pragma unroll
        for (int u = 0; u < ORB_UNITS; u++)   // A, row-major, from registers
            if (threadIdx.x + u * B < M2) s0[threadIdx.x + u * B] = av[u];
        __syncthreads();
        if (active) tile22(s1, s0, M, r, c, acc);   // T A
        __syncthreads();                            // every read of A done before R overwrites it
        if (active) {
            const float sc = (float)((ch == 0 ? 1.0 : 2.0) * scal[1]);   // c_P = 1, c_C = 2, times the output scale
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) s0[(r + i) * M + c + j] = make_float2(sc * acc[i][j].x, sc * acc[i][j].y);
        }
        __syncthreads();
    }
    // the orbit's matrices, (member k, entry i) advanced incrementally over nmem x M^2
    const int total = nmem * M2;
    int k = 0, i = threadIdx.x;
    while (i >= M2) {
        i -= M2;
        k++;
    }
    for (int base = threadIdx.x; base < total; base += ORB_UNITS * B) {
        int kk[ORB_UNITS], ii[ORB_UNITS], code[ORB_UNITS];
#pragma unroll
        for (int u = 0; u < ORB_UNITS; u++) {
            kk[u] = k;
            ii[u] = i;
            i += B;
            while (i >= M2) {
                i -= M2;
                k++;
            }
        }
#pragma unroll
        for (int u = 0; u < ORB_UNITS; u++) {
            const bool ok = on && base + u * B < total;
            const int e = ok ? s_e[kk[u]] : -1;
            code[u] = e >= 0 ? emap[((size_t)e * 2 + ch) * M2 + ii[u]] : ii[u] << 3;
        }
#pragma unroll
        for (int u = 0; u < ORB_UNITS; u++) {
            if (base + u * B >= total) break;
            float2 v = make_float2(0.f, 0.f);
            if (on) {
                const float2 w = s0[code[u] >> 3];
                const bool sw = code[u] & 4;
                v.x = __uint_as_float(__float_as_uint(sw ? w.y : w.x) ^ ((unsigned)(code[u] & 2) << 30));
                v.y = __uint_as_float(__float_as_uint(sw ? w.x : w.y) ^ ((unsigned)(code[u] & 1) << 31));
            }
            store_w(out + ((size_t)ch * Nq + s_q2[kk[u]]) * M2 + ii[u], v);
        }
    }
}

// Two-band bond sets (N_s^2 = 4, M = 4 N_ff): one CTA per (q, channel), one 4 x 4 output tile per
// thread (rows {2i, 2i+1, M/2 + 2i, M/2 + 2i + 1}, columns likewise).  Shared memory holds two
// M x M buffers: A transposed and L for T^T = L^T A^T, then A (reloaded, row-major) and T^T for
// c T A, so one wave of CTAs covers all transfer momenta.
template <typename R>
__global__ void __launch_bounds__(256) vlv_tiled_kernel(const typename cpx<R>::t *A, const typename cpx<R>::t *Lc,
                                                        const int *dij, int Nq, int M, int nff, int nd, int chmask,
                                                        const double *scal, const int *qlist, double2 *out)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *s0 = reinterpret_cast<C2 *>(smem_raw);   // A^T, then A
    C2 *s1 = s0 + M * M;                         // L, then T^T
    const int q = qlist ? qlist[blockIdx.x] : blockIdx.x, ch = blockIdx.y;
    const int M2 = M * M, h = M / 2, nt = h / 2;   // nt x nt threads own tiles
    double2 *o = out + ((size_t)ch * Nq + q) * M2;
    if (!((chmask >> ch) & 1)) {
        for (int i = threadIdx.x; i < M2; i += blockDim.x) o[i] = make_double2(0.0, 0.0);
        return;
    }
    const C2 *a = A + ((size_t)ch * Nq + q) * M2;
    const C2 *lc = Lc + ((size_t)ch * Nq + q) * nd * 16;
    // A^T and the expanded loop matrix L[(R1,a),(R2,b)] = Lc[d(R1 - R2)][a][b] (coalesced reads)
    {
        // (r, c) of i advanced incrementally (runtime integer division runs on this GPU's slow pipe)
        const int dr = blockDim.x / M, dc = blockDim.x - dr * M;
        int r = threadIdx.x / M, c = threadIdx.x - r * M;
        for (int i = threadIdx.x; i < M2; i += blockDim.x) {
            s0[c * M + r] = a[i];
            s1[i] = lc[(dij[(r >> 2) * nff + (c >> 2)] * 4 + (r & 3)) * 4 + (c & 3)];
            r += dr;
            c += dc;
            if (c >= M) {
                c -= M;
                r++;
            }
        }
    }
    __syncthreads();
    const int t = threadIdx.x;
    const bool active = t < nt * nt;
    const int r = 2 * (t / nt), c = 2 * (t % nt);
    C2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = mk(R(0), R(0));
    // T^T = L^T A^T: tile rows index columns of L, tile columns rows of A, so the tile is stored
    // row-major into T^T with consecutive lanes on consecutive addresses
    if (active) tile44(s1, s0, M, r, c, acc);
    __syncthreads();
    const int rows[4] = {r, r + 1, h + r, h + r + 1}, cols[4] = {c, c + 1, h + c, h + c + 1};
    if (active) {
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                s1[rows[i] * M + cols[j]] = acc[i][j];   // T^T[rows_i][cols_j] = T[cols_j][rows_i]
                acc[i][j] = mk(R(0), R(0));
            }
    }
    for (int i = threadIdx.x; i < M2; i += blockDim.x) s0[i] = a[i];   // A, row-major (L2-resident reread)
    __syncthreads();
    if (active) {
        const R sc = R((ch == 0 ? 1.0 : 2.0) * scal[1]);   // c_P = 1, c_C = 2, times the output scale
        tile44(s1, s0, M, r, c, acc);                      // c T A
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) store_c(o + rows[i] * M + cols[j], acc[i][j], sc);
    }
}

template <typename R>
__global__ void vlv_small_kernel(const typename cpx<R>::t *A, const typename cpx<R>::t *Lc, const int *dij, int Nq,
                                 int M, int nff, int ns2, int nd, int chmask, const double *scal, const int *qlist, double2 *out)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sA = reinterpret_cast<C2 *>(smem_raw);
    C2 *sL = sA + M * M;
    C2 *sT = sL + M * M;
    const int q = qlist ? qlist[blockIdx.x] : blockIdx.x, ch = blockIdx.y;
    const size_t M2 = (size_t)M * M;
    double2 *o = out + ((size_t)ch * Nq + q) * M2;
    if (!((chmask >> ch) & 1)) {
        for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) o[i] = make_double2(0.0, 0.0);
        return;
    }
    const C2 *a = A + ((size_t)ch * Nq + q) * M2;
    const C2 *lc = Lc + ((size_t)ch * Nq + q) * nd * ns2 * ns2;
    for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) {
        sA[i] = a[i];
        const int r = i / M, c = i % M;
        const int d = dij[(r / ns2) * nff + c / ns2];
        sL[i] = lc[((size_t)d * ns2 + r % ns2) * ns2 + c % ns2];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) {
        const int r = i / M, c = i % M;
        C2 acc = mk(R(0), R(0));
        for (int k = 0; k < M; k++) cfma(acc, sA[r * M + k], sL[k * M + c]);
        sT[i] = acc;
    }
    __syncthreads();
    const double sc = (ch == 0 ? 1.0 : 2.0) * scal[1];   // c_P = 1, c_C = 2, times the output scale
    for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) {
        const int r = i / M, c = i % M;
        C2 acc = mk(R(0), R(0));
        for (int k = 0; k < M; k++) cfma(acc, sT[r * M + k], sA[k * M + c]);
        o[i] = make_double2(sc * (double)acc.x, sc * (double)acc.y);
    }
}

}  // namespace

// Symmetric states: dX/dT(q') = W dX/dT(q) W^dagger for the non-representative momenta q' (W maps row
// r' to source row srow[r'] with i^qrow[r'], conjugated for time-reversed elements).  One CTA per
// (q', channel) walks the M^2 entries; the element's row tables sit in shared memory and the entry
// indices advance incrementally (blockDim = dr M + dc).
// (re, im) of a complex FP64 value times i^k, with the signs flipped on the bit patterns (integer operations)
__device__ __forceinline__ double2 times_i_pow(double2 v, int k)
{
    const long long sg = (long long)0x8000000000000000ull;
    const long long re = __double_as_longlong(v.x), im = __double_as_longlong(v.y);
    switch (k & 3) {
    case 0: return v;
    case 1: return make_double2(__longlong_as_double(im ^ sg), v.x);
    case 2: return make_double2(__longlong_as_double(re ^ sg), __longlong_as_double(im ^ sg));
    default: return make_double2(v.y, __longlong_as_double(re ^ sg));
    }
}

// dX/dT of the non-representative momenta from their representative's result: target entry (r, c) of momentum q2
// = i^(qt[r] - qt[c]) (conjugated for antiunitary elements) times source entry (srow[r], srow[c]).  One CTA per
// (momentum, channel); the momenta run orbit after orbit (order[]), so each representative's matrix is read from
// DRAM once and then from L2 for the rest of its orbit.
__global__ void __launch_bounds__(256) sym_scatter_kernel(double2 *out, int Nq, int M, int dr, int dc, const int2 *qmap,
                                                          const int *list, const int *order, const SymElem *elem,
                                                          const int *srow, const int *qrow)
{
    extern __shared__ int s_tab[];   // [M] source rows, [M] quarter turns
    const int q2 = order[blockIdx.x], ch = blockIdx.y;
    const int2 ie = qmap[q2];
    const int q = list[ie.x];
    if (q == q2) return;             // representatives hold their own result
    const int *sr = srow + ((size_t)ie.y * 2 + ch) * M, *qr = qrow + ((size_t)ie.y * 2 + ch) * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        s_tab[i] = sr[i];
        s_tab[M + i] = qr[i];
    }
    __syncthreads();
    const bool conj = elem[ie.y].conj;
    const double2 *src = out + ((size_t)ch * Nq + q) * M * M;
    double2 *dst = out + ((size_t)ch * Nq + q2) * M * M;
    const int M2 = M * M;
    int r = threadIdx.x / M, c = threadIdx.x - r * M;
    for (int t = threadIdx.x; t < M2; t += blockDim.x) {
        double2 v = src[(size_t)s_tab[r] * M + s_tab[c]];
        if (conj) v.y = __longlong_as_double(__double_as_longlong(v.y) ^ (long long)0x8000000000000000ull);
        dst[t] = times_i_pow(v, s_tab[M + r] - s_tab[M + c]);
        r += dr;
        c += dc;
        if (c >= M) { c -= M; r++; }
    }
}

// The same copy, orbit by orbit: one CTA per (representative, block of ORB_RB source rows, channel) reads its rows
// once into shared memory and writes the target rows of every other member of the orbit, row r = sinv[i] of member q2
// taking source row i: entry (r, c) = i^(qt[r] - qt[c]) (conjugated for antiunitary elements) times row i's entry
// srow[c].  Warp w writes the target row of source row i0 + w, its lanes on consecutive columns (coalesced); the
// member's column maps are staged in shared memory.  DRAM then sees each representative's matrix read once and every
// member's matrix written once.
constexpr int ORB_RB = 8;
__global__ void __launch_bounds__(32 * ORB_RB) sym_orbit_copy_kernel(double2 *out, int Nq, int M, const int2 *qmap,
                                                                     const int *list, const int *orb_ofs, const int *orb_q,
                                                                     const SymElem *elem, const int *srow, const int *sinv,
                                                                     const int *qrow)
{
    extern __shared__ double2 s_rows[];   // [ORB_RB][M] source rows, then [M] column sources, [M] quarter turns
    int *s_sr = reinterpret_cast<int *>(s_rows + (size_t)ORB_RB * M), *s_qr = s_sr + M;
    const int p = blockIdx.x, i0 = blockIdx.y * ORB_RB, ch = blockIdx.z;
    const int q = list[p], nr = min(ORB_RB, M - i0), w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t M2 = (size_t)M * M;
    const double2 *src = out + ((size_t)ch * Nq + q) * M2 + (size_t)i0 * M;
    for (int t = threadIdx.x; t < nr * M; t += blockDim.x) s_rows[t] = src[t];
    const long long sg = (long long)0x8000000000000000ull;
    for (int mi = orb_ofs[p]; mi < orb_ofs[p + 1]; mi++) {
        const int q2 = orb_q[mi];
        if (q2 == q) continue;
        const int e = qmap[q2].y;
        const bool conj = elem[e].conj;
        const size_t tab = ((size_t)e * 2 + ch) * M;
        __syncthreads();   // the previous member's maps are no longer read (and the rows have landed)
        for (int c = threadIdx.x; c < M; c += blockDim.x) {
            s_sr[c] = srow[tab + c];
            s_qr[c] = qrow[tab + c];
        }
        __syncthreads();
        if (w >= nr) continue;
        const int r = sinv[tab + i0 + w], qrr = s_qr[r];
        const double2 *row = s_rows + (size_t)w * M;
        double2 *d = out + ((size_t)ch * Nq + q2) * M2 + (size_t)r * M;
        for (int c = lane; c < M; c += 32) {
            double2 v = row[s_sr[c]];
            if (conj) v.y = __longlong_as_double(__double_as_longlong(v.y) ^ sg);
            d[c] = times_i_pow(v, qrr - s_qr[c]);
        }
    }
}

cudaError_t launch_sym_scatter(tufrg_model *m, double2 *d_out)
{
    PhaseScope ps(m, PH_SCATTER);
    const int threads = 256;
    if (m->d_sym_sinv && m->d_orb_ofs) {
        const size_t smem = sizeof(double2) * ORB_RB * m->M + 2 * sizeof(int) * m->M;
        if (smem > 48 * 1024)
            TUFRG_CUDA_TRY(cudaFuncSetAttribute(sym_orbit_copy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sym_orbit_copy_kernel<<<dim3(m->n_loop_q, (m->M + ORB_RB - 1) / ORB_RB, 2), 32 * ORB_RB, smem, m->stream>>>(
            d_out, m->Nq, m->M, m->d_qmap, m->d_loop_list, m->d_orb_ofs, m->d_orb_q, m->d_sym_elem, m->d_sym_srow,
            m->d_sym_sinv, m->d_sym_qrow);
        return cudaGetLastError();
    }
    sym_scatter_kernel<<<dim3(m->Nq, 2), threads, 2 * sizeof(int) * m->M, m->stream>>>(
        d_out, m->Nq, m->M, threads / m->M, threads % m->M, m->d_qmap, m->d_loop_list, m->d_orb_q, m->d_sym_elem,
        m->d_sym_srow, m->d_sym_qrow);
    return cudaGetLastError();
}

int orbit_max_size() { return ORB_MAX; }

bool orbit_products_supported(const tufrg_model *m)
{
    return m->ns == 2 && m->M <= 64 && m->M % 2 == 0 && m->precision != TUFRG_FP64;
}

cudaError_t launch_products_sym(tufrg_model *m, int channel_mask, double2 *d_out)
{
    if (!m->d_sym_emap) {
        TUFRG_CUDA_TRY(launch_vlv(m, m->d_A, channel_mask, d_out, m->d_loop_list, m->n_loop_q));
        return launch_sym_scatter(m, d_out);
    }
    const int M = m->M;
    const int threads = 1024;   // (M/2)^2 <= 1024 threads form the product; all of them write the orbit
    const size_t smem = 2 * sizeof(float2) * M * M;
    if (smem > 48 * 1024)
        TUFRG_CUDA_TRY(cudaFuncSetAttribute(vlv_orbit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhaseScope ps(m, PH_VLV);
    vlv_orbit_kernel<<<dim3(m->n_loop_q, 2), threads, smem, m->stream>>>(
        m->d_A32, m->d_Lc32, m->d_orb_lexp, m->Nq, M, m->nd, channel_mask, m->d_scal, m->d_loop_list, m->d_orb_ofs,
        m->d_orb_q, m->d_qmap, m->d_sym_emap, d_out);
    return cudaGetLastError();
}

cudaError_t launch_vlv(tufrg_model *m, const double2 *d_A, int channel_mask, double2 *d_out, const int *qlist, int nlist)
{
    const int M = m->M;
    if (tc_supported(m)) return launch_vlv_tc(m, channel_mask, d_out, qlist, nlist);
    if (M > 64) return launch_vlv_large(m, d_A, channel_mask, d_out, qlist, nlist);
    const int ns2 = m->ns * m->ns;
    dim3 grid(qlist ? nlist : m->Nq, 2);
    PhaseScope ps(m, PH_VLV);
    if (ns2 == 4) {
        const int threads = std::max(32, ((M / 4) * (M / 4) + 31) / 32 * 32);   // <= 256 for M <= 64
        if (m->precision == TUFRG_FP64) {
            const size_t smem = 2 * sizeof(double2) * M * M;
            auto k = vlv_tiled_kernel<double>;
            if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k<<<grid, threads, smem, m->stream>>>(d_A, m->d_Lc, m->d_dij, m->Nq, M, m->nff, m->nd, channel_mask,
                                                  m->d_scal, qlist, d_out);
        } else {
            const size_t smem = 2 * sizeof(float2) * M * M;
            auto k = vlv_tiled_kernel<float>;
            if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k<<<grid, threads, smem, m->stream>>>(m->d_A32, m->d_Lc32, m->d_dij, m->Nq, M, m->nff, m->nd, channel_mask,
                                                  m->d_scal, qlist, d_out);
        }
        return cudaGetLastError();
    }
    const int threads = 256;
    if (m->precision == TUFRG_FP64) {
        const size_t smem = 3 * sizeof(double2) * M * M;
        auto k = vlv_small_kernel<double>;
        if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, threads, smem, m->stream>>>(d_A, m->d_Lc, m->d_dij, m->Nq, M, m->nff, ns2, m->nd, channel_mask,
                                              m->d_scal, qlist, d_out);
    } else {
        const size_t smem = 3 * sizeof(float2) * M * M;
        auto k = vlv_small_kernel<float>;
        if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, threads, smem, m->stream>>>(m->d_A32, m->d_Lc32, m->d_dij, m->Nq, M, m->nff, ns2, m->nd,
                                              channel_mask, m->d_scal, qlist, d_out);
    }
    return cudaGetLastError();
}

}  // namespace tufrg
