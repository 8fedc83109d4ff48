// Channel projections of Sec. 3.3 on the device.
//
//   X(R'') = (1/Nq) sum_u e^{i u.R''} X(u)                         (Fourier transform, after Eq. zw_1)
//   A_P = P^[V0] + P + P^[V^C] + P^[V^D]                            (Eq. sum_P)
//     P^[V^C]_{RR'}(s) =  sum_R'' e^{i s.R''} C^{R+R'',R'-R''}_{s1s2s3s4}(R'')        (Eq. proj_PD)
//     P^[V^D]_{RR'}(s) = -e^{i s.R'} sum_R'' e^{i s.R''} C^{R+R'',-R'-R''}_{s1s2s4s3}(R'')
//   A_C = C^[V0] + C^[V^P] + C + C^[V^D]
//     C^[V^P]_{RR'}(u) =  sum_R'' e^{i u.R''} P^{R+R'',R'-R''}_{s1s2s3s4}(R'')
//     C^[V^D]_{RR'}(u) = -sum_R'' e^{i u.R''} C^{R-R'+R'',R''}_{s1s2s4s3}(-R')        (Eq. proj_DC)
//
// Fourier transform: one thread per matrix entry and a slice of the transfer mesh,
// a block of bond classes in registers, phases staged in shared memory; the
// slices are added in a fixed order by a second kernel (deterministic).  The
// state is read once from HBM; the split path accumulates in FP32.
//
// Projections: the bond arithmetic is done once on the host into int32 gather
// tables, flattened per output matrix entry: each term is the flat index of its
// source in the Fourier transforms (sign in the high bit) and a phase-table column.
// A thread owns one matrix entry and QT transfer momenta: it walks its term list
// once, each source value (independent of q) is loaded once and applied with the
// QT momenta's phases from shared memory, and the state is read and the result
// written fully coalesced.  max |A| is reduced in the CTA and merged with one
// atomic per CTA.  The split path reads the FP32 copy of the state.
#include <algorithm>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

template <typename R> __device__ __forceinline__ typename cpx<R>::t ld_as(const double2 &v);
template <> __device__ __forceinline__ double2 ld_as<double>(const double2 &v) { return v; }
// FP64 -> FP32 of a complex value: the real part by the hardware conversion (the FP64 pipe), the imaginary part on
// the integer pipe (narrow_f, the same rounding bit for bit), so that the two pipes share the work
template <> __device__ __forceinline__ float2 ld_as<float>(const double2 &v) { return make_float2(__double2float_rn(v.x), narrow_f(v.y)); }
template <typename R> __device__ __forceinline__ typename cpx<R>::t ld_as(const float2 &v);
template <> __device__ __forceinline__ float2 ld_as<float>(const float2 &v) { return v; }

template <typename R, typename XT, int CPT>
__global__ void __launch_bounds__(128) dft_kernel(const XT *__restrict__ X, int Nq, int M2, int ncls, int nchunk,
                                                  const XT *__restrict__ clsph, int u_per,
                                                  typename cpx<R>::t *__restrict__ part)
{
    using C2 = typename cpx<R>::t;
    constexpr int UB = 8;   // loads in flight per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *ph = reinterpret_cast<C2 *>(smem_raw);   // [u_per][CPT]
    const int ch = blockIdx.z / nchunk, c0 = (blockIdx.z % nchunk) * CPT;
    const int u0 = blockIdx.y * u_per, u1 = min(Nq, u0 + u_per);
    for (int i = threadIdx.x; i < (u1 - u0) * CPT; i += blockDim.x) {
        const int u = u0 + i / CPT, c = c0 + i % CPT;
        ph[i] = c < ncls ? ld_as<R>(clsph[(size_t)u * ncls + c]) : mk(R(0), R(0));
    }
    __syncthreads();
    const int ij = blockIdx.x * blockDim.x + threadIdx.x;
    if (ij >= M2) return;
    C2 acc[CPT];
#pragma unroll
    for (int c = 0; c < CPT; c++) acc[c] = mk(R(0), R(0));
    const XT *src = X + ((size_t)ch * Nq + u0) * M2 + ij;
    int u = u0;
    for (; u + UB <= u1; u += UB, src += (size_t)UB * M2) {
        C2 x[UB];
#pragma unroll
        for (int j = 0; j < UB; j++) x[j] = ld_as<R>(src[(size_t)j * M2]);
#pragma unroll
        for (int j = 0; j < UB; j++) {
            const C2 *p = ph + (u + j - u0) * CPT;
#pragma unroll
            for (int c = 0; c < CPT; c++) {
                acc[c].x = fma(p[c].x, x[j].x, fma(-p[c].y, x[j].y, acc[c].x));
                acc[c].y = fma(p[c].x, x[j].y, fma(p[c].y, x[j].x, acc[c].y));
            }
        }
    }
    for (; u < u1; u++, src += M2) {
        const C2 x = ld_as<R>(*src);
        const C2 *p = ph + (u - u0) * CPT;
#pragma unroll
        for (int c = 0; c < CPT; c++) {
            acc[c].x = fma(p[c].x, x.x, fma(-p[c].y, x.y, acc[c].x));
            acc[c].y = fma(p[c].x, x.y, fma(p[c].y, x.x, acc[c].y));
        }
    }
#pragma unroll
    for (int c = 0; c < CPT; c++)
        if (c0 + c < ncls) part[(((size_t)blockIdx.y * 2 + ch) * ncls + c0 + c) * M2 + ij] = acc[c];
}

// Separable form of the same transform, u = (u_x, u_y), R'' = (R_x, R_y):
//   Z(u_x, R_y) = sum_{u_y} e^{i u_y R_y} X(u_x, u_y),   X(R'') = (1/Nq) sum_{u_x} e^{i u_x R_x} Z(u_x, R_y),
// Lq (n_Ry + n_cls / Lq) complex FMAs per entry and class instead of Nq, in two passes:
//   dft_rows_kernel: one thread per (channel, u_x, matrix entry) reads its Lq values of the state, UB loads in
//     flight at a time (the only pass over the state, coalesced across entries), keeps Z for the n_Ry distinct
//     R_y of the classes in registers and writes them to a scratch [ch][u_x][R_y][M^2] (n_Ry / Lq of the state's
//     size: 2.5 MB at the 24x24 two-band workload, held in L2); reading the FP64 state on the split path it also
//     writes the FP32 rounding (the copy the projections read);
//   dft_cols_kernel: a CTA per (channel, R_y, 32 consecutive entries) stages Z(u_x, R_y) of its entries in shared
//     memory, DFT_UXC values of u_x at a time; warp w adds e^{i u_x R_x} Z(u_x, R_y) over u_x for the w-th class
//     with that R_y, one entry per lane.
// Both sums run in a fixed order (deterministic).  Neither kernel holds partial sums of the classes in shared
// memory, so their CTAs are small and share the SMs with the loop k-sum that runs beside the state's branch.
constexpr int DFT_MAXRY = 9;
constexpr int DFT_MAXG = 32;     // classes of one R_y (warps of a dft_cols_kernel CTA)
constexpr int DFT_UXC = 32;      // u_x staged per round in dft_cols_kernel
constexpr int DFT_THREADS = 128;
constexpr size_t DFT_TABLE_CAP = 32 * 1024;   // phases (and class tables) staged in shared memory

__device__ __forceinline__ void put32(float2 *p, float2 v) { *p = v; }
__device__ __forceinline__ void put32(float2 *, double2) {}

template <typename R, typename XT>
__global__ void __launch_bounds__(DFT_THREADS) dft_rows_kernel(const XT *__restrict__ X, int Lq, int M2, int nry,
                                                               const typename cpx<R>::t *__restrict__ phy, int ch_lo,
                                                               typename cpx<R>::t *__restrict__ Z,
                                                               float2 *__restrict__ x32)
{
    using C2 = typename cpx<R>::t;
    constexpr int UB = 8;   // loads in flight per thread (more registers than this leave too few warps per SM)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sphy = reinterpret_cast<C2 *>(smem_raw);   // [Lq][nry]  e^{i u_y R_y}
    for (int i = threadIdx.x; i < Lq * nry; i += blockDim.x) sphy[i] = phy[i];
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + threadIdx.x, ux = blockIdx.y, ch = ch_lo + blockIdx.z;
    if (e >= M2) return;
    const size_t row = ((size_t)ch * Lq * Lq + (size_t)ux * Lq) * M2 + e;
    C2 z[DFT_MAXRY];
#pragma unroll
    for (int r = 0; r < DFT_MAXRY; r++) z[r] = mk(R(0), R(0));
    for (int uy0 = 0; uy0 < Lq; uy0 += UB) {
        // all loads of the batch first, then the roundings (and the FP32 copy)
        XT raw[UB];
#pragma unroll
        for (int j = 0; j < UB; j++) {
            raw[j].x = 0;
            raw[j].y = 0;
            if (uy0 + j < Lq) raw[j] = X[row + (size_t)(uy0 + j) * M2];
        }
        C2 x[UB];
#pragma unroll
        for (int j = 0; j < UB; j++) {
            x[j] = ld_as<R>(raw[j]);
            if (x32 && uy0 + j < Lq) put32(x32 + row + (size_t)(uy0 + j) * M2, x[j]);
        }
#pragma unroll
        for (int j = 0; j < UB; j++) {
            if (uy0 + j >= Lq) break;
            const C2 *p = sphy + (uy0 + j) * nry;
#pragma unroll
            for (int r = 0; r < DFT_MAXRY; r++) {
                if (r >= nry) break;
                const C2 ph = p[r];
                z[r].x = fma(ph.x, x[j].x, fma(-ph.y, x[j].y, z[r].x));
                z[r].y = fma(ph.x, x[j].y, fma(ph.y, x[j].x, z[r].y));
            }
        }
    }
    C2 *zo = Z + ((size_t)ch * Lq + ux) * nry * M2 + e;
#pragma unroll
    for (int r = 0; r < DFT_MAXRY; r++)
        if (r < nry) zo[(size_t)r * M2] = z[r];
}

// Classes are visited grouped by R_y: sorted position c has class id cid[c] and R_x index rxi[c], and the group of
// the r-th R_y is [ryo[r], ryo[r+1]).
template <typename R>
__global__ void __launch_bounds__(32 * DFT_MAXG) dft_cols_kernel(const typename cpx<R>::t *__restrict__ Z, int Lq,
                                                                 int M2, int ncls, int nry, int nrx,
                                                                 const int *__restrict__ tabs,
                                                                 const typename cpx<R>::t *__restrict__ phx, int ch_lo,
                                                                 double inv_nq, typename cpx<R>::t *__restrict__ Xr)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sz = reinterpret_cast<C2 *>(smem_raw);              // [DFT_UXC][32]  Z(u_x, R_y) of the CTA's entries
    C2 *sphx = sz + DFT_UXC * 32;                           // [Lq][nrx]  e^{i u_x R_x}
    int *stab = reinterpret_cast<int *>(sphx + Lq * nrx);   // cid [ncls], rxi [ncls], ryo [nry + 1]
    for (int i = threadIdx.x; i < Lq * nrx; i += blockDim.x) sphx[i] = phx[i];
    for (int i = threadIdx.x; i < 2 * ncls + nry + 1; i += blockDim.x) stab[i] = tabs[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e0 = blockIdx.x * 32, r = blockIdx.y, ch = ch_lo + blockIdx.z;
    const int *cid = stab, *rxi = stab + ncls, *ryo = stab + 2 * ncls;
    const int c = ryo[r] + w;
    const bool mine = c < ryo[r + 1];   // this warp's class (warps past the group only help stage Z)
    const int rx = mine ? rxi[c] : 0;
    const C2 *zc = Z + ((size_t)ch * Lq * nry + r) * M2 + e0;   // Z(u_x, R_y) of entry e0 + l at zc[u_x nry M^2 + l]
    const size_t zs = (size_t)nry * M2;
    const int ne = min(32, M2 - e0);
    C2 acc = mk(R(0), R(0));
    for (int u0 = 0; u0 < Lq; u0 += DFT_UXC) {
        const int nu = min(DFT_UXC, Lq - u0);
        __syncthreads();   // the previous round's reads are done
        for (int i = threadIdx.x; i < nu * 32; i += blockDim.x) {
            const int ul = i >> 5, l = i & 31;
            sz[i] = l < ne ? zc[(size_t)(u0 + ul) * zs + l] : mk(R(0), R(0));
        }
        __syncthreads();
        if (mine)
            for (int ul = 0; ul < nu; ul++) {
                const C2 v = sz[ul * 32 + lane];
                const C2 ph = sphx[(u0 + ul) * nrx + rx];
                acc.x = fma(ph.x, v.x, fma(-ph.y, v.y, acc.x));
                acc.y = fma(ph.x, v.y, fma(ph.y, v.x, acc.y));
            }
    }
    if (mine && lane < ne) {
        const R scale = R(inv_nq);
        Xr[((size_t)ch * ncls + cid[c]) * M2 + e0 + lane] = mk(acc.x * scale, acc.y * scale);
    }
}

template <typename R>
__global__ void dft_reduce_kernel(const typename cpx<R>::t *part, int nsplit, int ch_lo, int nch, int ncls, int M2,
                                  double inv_nq, typename cpx<R>::t *Xr)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // over nch * ncls * M2
    const size_t per = (size_t)ncls * M2;
    if (i >= (size_t)nch * per) return;
    const int ch = ch_lo + (int)(i / per);
    const size_t r = i % per;
    R sx = 0, sy = 0;
    for (int s = 0; s < nsplit; s++) {
        const auto v = part[((size_t)s * 2 + ch) * per + r];
        sx += v.x;
        sy += v.y;
    }
    Xr[(size_t)ch * per + r] = mk(R(sx * inv_nq), R(sy * inv_nq));
}

// |v|^2 with one explicit rounding order, shared by the projection and the arg-max search so that
// both see the same bits
__device__ __forceinline__ double abs2(double2 v) { return fma(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ float abs2(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }
// max |A| as the double that the flow controller reads
__device__ __forceinline__ double mag_of(double m2) { return sqrt(m2); }
__device__ __forceinline__ double mag_of(float m2) { return (double)sqrtf(m2); }

// Projected vertices A_X(q) for QT transfer momenta of one channel, one matrix entry per thread.
// The plain path works in FP64; the split path forms A in FP32 (its only consumer is the FP32 V.L.V
// product) and writes the FP64 copy only when asked (A != NULL).
template <typename R, typename XT, int QT>
__global__ void __launch_bounds__(256) project_kernel(const XT *__restrict__ X, const typename cpx<R>::t *__restrict__ Xr,
                                                      const XT *v0d0, const XT *v0d1, const int *eofs0,
                                                      const int *eofs1, const int2 *et0, const int2 *et1,
                                                      const typename cpx<R>::t *ph, int nph, int Nq, int M2, int ncls,
                                                      int chmask, const int *qlist, int nlist, double2 *A, float2 *A32,
                                                      unsigned long long *amax, int x_local, const XT *v0q)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *phs = reinterpret_cast<C2 *>(smem_raw);   // [QT][nph]
    __shared__ int sq[QT];                         // transfer momenta of this CTA (list positions p0 ..)
    const int ch = blockIdx.z, p0 = blockIdx.y * QT, nq = min(QT, nlist - p0);
    if (threadIdx.x < QT) sq[threadIdx.x] = threadIdx.x < nq ? (qlist ? qlist[p0 + threadIdx.x] : p0 + threadIdx.x) : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < QT * nph; i += blockDim.x) {
        const int qi = i / nph;
        phs[i] = qi < nq ? ph[(size_t)sq[qi] * nph + (i - qi * nph)] : mk(R(0), R(0));
    }
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    R m2 = R(0);
    if (e < M2) {
        const bool on = (chmask >> ch) & 1;
        const size_t base = (size_t)ch * Nq * M2 + e;   // + q M2
        // the state rows: at their momenta, or (x_local) in list order, [2][nlist][M2]
        const size_t xbase = x_local ? ((size_t)ch * nlist + p0) * M2 + e : base;
        C2 acc[QT];
        if (on) {
            const C2 v0 = ld_as<R>((ch == 0 ? v0d0 : v0d1)[e]);
#pragma unroll
            for (int qi = 0; qi < QT; qi++) {
                acc[qi] = qi < nq ? ld_as<R>(X[xbase + (size_t)(x_local ? qi : sq[qi]) * M2]) : mk(R(0), R(0));
                // the bare vertex: onsite (one value for every momentum), or per momentum in the band basis
                const C2 vq = v0q && qi < nq ? ld_as<R>(v0q[((size_t)ch * Nq + sq[qi]) * M2 + e]) : v0;
                acc[qi].x += vq.x;
                acc[qi].y += vq.y;
            }
            const int *eofs = ch == 0 ? eofs0 : eofs1;
            const int2 *et = ch == 0 ? et0 : et1;
            const int t1 = eofs[e + 1];
            const int lim = ncls * M2;   // sources at or above lim belong to the C channel
            // TB terms per iteration: every term's gathers are issued before any is used (the terms are
            // still added in their order)
            constexpr int TB = 4;
            int t = eofs[e];
            for (; t + TB <= t1; t += TB) {
                int2 g[TB];
                C2 x[TB];
#pragma unroll
                for (int j = 0; j < TB; j++) g[j] = et[t + j];
#pragma unroll
                for (int j = 0; j < TB; j++) {
                    const int idx = g[j].x & 0x7fffffff;
                    x[j] = ((chmask >> (idx >= lim ? 1 : 0)) & 1) ? Xr[idx] : mk(R(0), R(0));
                }
#pragma unroll
                for (int j = 0; j < TB; j++) {
                    if (g[j].x < 0) { x[j].x = -x[j].x; x[j].y = -x[j].y; }
                    const C2 *pj = phs + g[j].y;
#pragma unroll
                    for (int qi = 0; qi < QT; qi++) {
                        const C2 pq = pj[qi * nph];
                        acc[qi].x += pq.x * x[j].x - pq.y * x[j].y;
                        acc[qi].y += pq.x * x[j].y + pq.y * x[j].x;
                    }
                }
            }
            for (; t < t1; t++) {
                const int2 g = et[t];
                const int idx = g.x & 0x7fffffff;
                if ((chmask >> (idx >= lim ? 1 : 0)) & 1) {
                    C2 x = Xr[idx];
                    if (g.x < 0) { x.x = -x.x; x.y = -x.y; }
                    const C2 *p = phs + g.y;
#pragma unroll
                    for (int qi = 0; qi < QT; qi++) {
                        const C2 pq = p[qi * nph];
                        acc[qi].x += pq.x * x.x - pq.y * x.y;
                        acc[qi].y += pq.x * x.y + pq.y * x.x;
                    }
                }
            }
        } else {
#pragma unroll
            for (int qi = 0; qi < QT; qi++) acc[qi] = mk(R(0), R(0));
        }
#pragma unroll
        for (int qi = 0; qi < QT; qi++) {
            if (qi >= nq) break;
            const size_t o = base + (size_t)sq[qi] * M2;
            if (A) A[o] = make_double2((double)acc[qi].x, (double)acc[qi].y);
            if (A32) A32[o] = make_float2((float)acc[qi].x, (float)acc[qi].y);
            m2 = max(m2, abs2(acc[qi]));
        }
    }
    // max |A| over the CTA, then one atomic (non-negative doubles order like their bit patterns)
    __shared__ R wmax[8];
    for (int off = 16; off > 0; off >>= 1) m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, off));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) m2 = max(m2, wmax[w]);
        if (m2 > R(0)) atomicMax(amax, (unsigned long long)__double_as_longlong(mag_of(m2)));
    }
}

// Locate the maximum: every entry whose magnitude equals the reduced maximum records its flat index
// (atomicMin keeps the first).  The magnitude is formed exactly as in the projection.
// With qmap / list (projections of orbit representatives only) other momenta hold stale values and are skipped.
template <typename C2>
__global__ void amax_locate_kernel(const C2 *A, size_t n, const unsigned long long *amax, unsigned long long *where,
                                   const int2 *qmap, const int *list, size_t M2, int Nq)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (qmap) {
        const int q = (int)((i / M2) % (size_t)Nq);
        if (list[qmap[q].x] != q) return;
    }
    if ((unsigned long long)__double_as_longlong(mag_of(abs2(A[i]))) == *amax) atomicMin(where, (unsigned long long)i);
}

// max |A| per channel (out[0] = P, out[1] = C, bit patterns of the non-negative magnitudes, atomicMax), the
// magnitude formed as in the projection; grid-stride, one atomic per warp and channel run
template <typename C2>
__global__ void __launch_bounds__(256) amax_channels_kernel(const C2 *A, size_t n, unsigned long long *out,
                                                            const int2 *qmap, const int *list, size_t M2, int Nq)
{
    const size_t per_ch = M2 * (size_t)Nq;
    unsigned long long best[2] = {0ull, 0ull};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (qmap) {
            const int q = (int)((i / M2) % (size_t)Nq);
            if (list[qmap[q].x] != q) continue;
        }
        const unsigned long long b = (unsigned long long)__double_as_longlong(mag_of(abs2(A[i])));
        const int ch = i < per_ch ? 0 : 1;
        best[ch] = b > best[ch] ? b : best[ch];
    }
#pragma unroll
    for (int ch = 0; ch < 2; ch++) {
        unsigned long long v = best[ch];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if ((threadIdx.x & 31) == 0 && v) atomicMax(out + ch, v);
    }
}

template <typename R, typename XT, int CPT>
cudaError_t dft_run(tufrg_model *m, const XT *d_state, const XT *clsph, int ch_lo, int nch, typename cpx<R>::t *part,
                    typename cpx<R>::t *Xr)
{
    const int M2 = m->M * m->M;
    const int threads = 128;
    const int nchunk = (m->ncls + CPT - 1) / CPT;
    const int xb = (M2 + threads - 1) / threads;
    const int nsplit = m->dft_nsplit;
    const int u_per = (m->Nq + nsplit - 1) / nsplit;
    const size_t smem = sizeof(typename cpx<R>::t) * u_per * CPT;
    auto k = dft_kernel<R, XT, CPT>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        PhaseScope ps(m, PH_DFT, 2);
        dim3 grid(xb, nsplit, nch * nchunk);
        // channels are numbered from ch_lo inside the kernels
        k<<<grid, threads, smem, m->stream>>>(d_state + (size_t)ch_lo * m->Nq * M2, m->Nq, M2, m->ncls, nchunk, clsph,
                                               u_per, part);
        TUFRG_CUDA_TRY(cudaGetLastError());
        const size_t total = (size_t)nch * m->ncls * M2;
        dft_reduce_kernel<R><<<(unsigned)((total + 255) / 256), 256, 0, m->stream>>>(
            part, nsplit, 0, nch, m->ncls, M2, 1.0 / m->Nq, Xr + (size_t)ch_lo * m->ncls * M2);
    }
    return cudaGetLastError();
}

}  // namespace

int dft_plan_nsplit(const tufrg_model *m)
{
    const int xb = (m->M * m->M + 127) / 128;
    const int cpt = m->precision == TUFRG_FP64 ? 16 : 32;
    const int nchunk = (m->ncls + cpt - 1) / cpt;
    const long want = 4L * m->sm_count;
    long ns = (want + (long)xb * 2 * nchunk - 1) / ((long)xb * 2 * nchunk);
    // the phases of a CTA's slice of the transfer mesh must fit in 96 KB of shared memory
    const long esize = m->precision == TUFRG_FP64 ? 16 : 8;
    const long cap = 96L * 1024 / (cpt * esize);
    ns = std::max(ns, ((long)m->Nq + cap - 1) / cap);
    if (ns < 1) ns = 1;
    if (ns > m->Nq) ns = m->Nq;
    return (int)ns;
}

// whether the separable transform applies (*warps = warps of a dft_cols_kernel CTA = the largest number of classes
// with one R_y, 0: the sliced direct sum runs instead): at most DFT_MAXRY distinct R_y, at most DFT_MAXG classes per
// R_y, and the phase and class tables of each kernel within DFT_TABLE_CAP
void dft_sep_plan(const tufrg_model *m, int *warps)
{
    *warps = 0;
    if (m->dft_nry < 1 || m->dft_nry > DFT_MAXRY) return;
    const size_t c2 = m->precision == TUFRG_FP64 ? sizeof(double2) : sizeof(float2);
    if (c2 * m->Lq * m->dft_nry > DFT_TABLE_CAP) return;
    if (c2 * (m->Lq * m->dft_nrx + DFT_UXC * 32) + sizeof(int) * (2 * m->ncls + m->dft_nry + 1) > DFT_TABLE_CAP) return;
    int gmax = 0;
    for (int c = 0; c < m->ncls; c++) {
        int g = 0;
        for (int c2 = 0; c2 < m->ncls; c2++) g += m->cls[2 * c2 + 1] == m->cls[2 * c + 1];
        gmax = std::max(gmax, g);
    }
    if (gmax < 1 || gmax > DFT_MAXG) return;
    *warps = gmax;
}

template <typename R, typename XT>
cudaError_t dft_sep_run(tufrg_model *m, const XT *d_state, const typename cpx<R>::t *phy, const typename cpx<R>::t *phx,
                        int ch_lo, int nch, typename cpx<R>::t *Xr, float2 *x32)
{
    using C2 = typename cpx<R>::t;
    const int M2 = m->M * m->M, xb = (M2 + DFT_THREADS - 1) / DFT_THREADS;
    C2 *Z = static_cast<C2 *>(m->d_dftpart);
    const size_t smem_rows = sizeof(C2) * (size_t)m->Lq * m->dft_nry;
    const size_t smem_cols = sizeof(C2) * ((size_t)m->Lq * m->dft_nrx + DFT_UXC * 32) +
                             sizeof(int) * (2 * m->ncls + m->dft_nry + 1);
    PhaseScope ps(m, PH_DFT, 2);
    dft_rows_kernel<R, XT><<<dim3(xb, m->Lq, nch), DFT_THREADS, smem_rows, m->stream>>>(d_state, m->Lq, M2, m->dft_nry, phy, ch_lo, Z,
                                                                      x32);
    TUFRG_CUDA_TRY(cudaGetLastError());
    dft_cols_kernel<R><<<dim3((M2 + 31) / 32, m->dft_nry, nch), 32 * m->dft_warps, smem_cols, m->stream>>>(
        Z, m->Lq, M2, m->ncls, m->dft_nry, m->dft_nrx, m->d_dft_tabs, phx, ch_lo, 1.0 / m->Nq, Xr);
    return cudaGetLastError();
}

cudaError_t launch_dft(tufrg_model *m, const double2 *d_state, const float2 *d_state32, int channel_mask)
{
    const int ch_lo = (channel_mask & 1) ? 0 : 1, ch_hi = (channel_mask & 2) ? 1 : 0;
    if (ch_lo > ch_hi) return cudaSuccess;
    const int nch = ch_hi - ch_lo + 1;
    if (m->dft_warps > 0) {
        if (m->precision == TUFRG_FP64)
            return dft_sep_run<double, double2>(m, d_state, m->d_dft_phy, m->d_dft_phx, ch_lo, nch, m->d_Xr, nullptr);
        // the split path reads the FP32 copy where one exists, else the FP64 state, writing its rounding to
        // the model's copy as it reads
        if (d_state32)
            return dft_sep_run<float, float2>(m, d_state32, m->d_dft_phy32, m->d_dft_phx32, ch_lo, nch, m->d_Xr32,
                                              nullptr);
        return dft_sep_run<float, double2>(m, d_state, m->d_dft_phy32, m->d_dft_phx32, ch_lo, nch, m->d_Xr32, m->d_X32);
    }
    if (m->precision == TUFRG_FP64)
        return dft_run<double, double2, 16>(m, d_state, m->d_clsph, ch_lo, nch, reinterpret_cast<double2 *>(m->d_dftpart),
                                            m->d_Xr);
    if (!d_state32) return cudaErrorInvalidValue;   // callers convert first when the separable form does not apply
    return dft_run<float, float2, 32>(m, d_state32, m->d_clsph32, ch_lo, nch, reinterpret_cast<float2 *>(m->d_dftpart),
                                      m->d_Xr32);
}

constexpr int PROJ_QT = 8;   // transfer momenta per thread

// FP64 tables on the plain path, their FP32 copies on the split path (where d_A may be NULL)
template <typename R, typename XT, int QT>
cudaError_t project_run(tufrg_model *m, const XT *d_state, const typename cpx<R>::t *Xr, const XT *v0d0, const XT *v0d1,
                        const typename cpx<R>::t *ph, int channel_mask, const int *qlist, int nlist, double2 *d_A,
                        float2 *d_A32, int x_local, const XT *v0q)
{
    const int M2 = m->M * m->M;
    const dim3 grid((M2 + 255) / 256, (nlist + QT - 1) / QT, 2);
    const size_t smem = sizeof(typename cpx<R>::t) * QT * m->nph;
    auto k = project_kernel<R, XT, QT>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<grid, 256, smem, m->stream>>>(d_state, Xr, v0d0, v0d1, m->d_eofs[0], m->d_eofs[1], m->d_eterms[0],
                                      m->d_eterms[1], ph, m->nph, m->Nq, M2, m->ncls, channel_mask, qlist, nlist, d_A,
                                      d_A32, m->d_amax, x_local, v0q);
    return cudaGetLastError();
}

cudaError_t launch_project(tufrg_model *m, const double2 *d_state, const float2 *d_state32, int channel_mask,
                           double2 *d_A, const int *qlist, int nlist)
{
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax, 0, sizeof(unsigned long long), m->stream));
    const int M2 = m->M * m->M;
    if (!qlist) nlist = m->Nq;
    const int xb = (M2 + 255) / 256;
    // QT momenta share each gathered source value; a short list (orbit representatives) takes QT = 2 so
    // that its grid still covers the GPU
    const bool short_list = (long)((nlist + PROJ_QT - 1) / PROJ_QT) * xb * 2 < 2L * m->sm_count;
    PhaseScope ps(m, PH_PROJ);
    if (m->precision == TUFRG_FP64) {
        auto run = short_list ? project_run<double, double2, 2> : project_run<double, double2, PROJ_QT>;
        return run(m, d_state, m->d_Xr, m->d_v0d[0], m->d_v0d[1], m->d_ph, channel_mask, qlist, nlist, d_A, nullptr, 0,
                   m->d_v0q);
    }
    if (!d_state32) return cudaErrorInvalidValue;   // the split path projects the FP32 copy
    auto run = short_list ? project_run<float, float2, 2> : project_run<float, float2, PROJ_QT>;
    return run(m, d_state32, m->d_Xr32, m->d_v0d32[0], m->d_v0d32[1], m->d_ph32, channel_mask, qlist, nlist, d_A,
               m->d_A32, 0, m->d_v0q32);
}

cudaError_t launch_project_local(tufrg_model *m, const double2 *d_state_local, const float2 *d_state32_local,
                                 int channel_mask, double2 *d_A, const int *qlist, int nlist)
{
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax, 0, sizeof(unsigned long long), m->stream));
    PhaseScope ps(m, PH_PROJ);
    if (m->precision == TUFRG_FP64)
        return project_run<double, double2, 2>(m, d_state_local, m->d_Xr, m->d_v0d[0], m->d_v0d[1], m->d_ph, channel_mask,
                                               qlist, nlist, d_A, nullptr, 1, m->d_v0q);
    return project_run<float, float2, 2>(m, d_state32_local, m->d_Xr32, m->d_v0d32[0], m->d_v0d32[1], m->d_ph32,
                                         channel_mask, qlist, nlist, d_A, m->d_A32, 1, m->d_v0q32);
}

cudaError_t launch_amax_channels(tufrg_model *m, bool reps_only)
{
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax_ch, 0, 2 * sizeof(unsigned long long), m->stream));
    m->launches++;
    const size_t n = 2 * (size_t)m->Nq * m->M * m->M, M2 = (size_t)m->M * m->M;
    const int2 *qm = reps_only ? m->d_qmap : nullptr;
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)m->sm_count * 8);
    if (m->precision == TUFRG_FP64)
        amax_channels_kernel<<<grid, 256, 0, m->stream>>>(m->d_A, n, m->d_amax_ch, qm, m->d_loop_list, M2, m->Nq);
    else
        amax_channels_kernel<<<grid, 256, 0, m->stream>>>(m->d_A32, n, m->d_amax_ch, qm, m->d_loop_list, M2, m->Nq);
    return cudaGetLastError();
}

cudaError_t launch_amax_locate(tufrg_model *m, size_t n, bool reps_only)
{
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax + 1, 0xff, sizeof(unsigned long long), m->stream));
    m->launches++;
    const unsigned grid = (unsigned)((n + 255) / 256);
    const int2 *qm = reps_only ? m->d_qmap : nullptr;
    const size_t M2 = (size_t)m->M * m->M;
    if (m->precision == TUFRG_FP64)
        amax_locate_kernel<<<grid, 256, 0, m->stream>>>(m->d_A, n, m->d_amax, m->d_amax + 1, qm, m->d_loop_list, M2, m->Nq);
    else
        amax_locate_kernel<<<grid, 256, 0, m->stream>>>(m->d_A32, n, m->d_amax, m->d_amax + 1, qm, m->d_loop_list, M2, m->Nq);
    return cudaGetLastError();
}

}  // namespace tufrg
