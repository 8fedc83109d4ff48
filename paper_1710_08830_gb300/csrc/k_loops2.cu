// Split-precision (FP32) loop k-sum for N_s = 2, the dominant kernel of the right-hand side.
//
// Same sums as k_loops.cu (Eqs. loopminus / loopplus dressed by Eq. trafo), organised
// around the structure of the two-band problem:
//   * the band projectors are complete and rank one: rho^1 = 1 - rho^0 and
//     rho^0_00 + rho^0_11 = 1, so one 48-byte record per fine k holds
//     (rho^0_00, Re rho^0_01, Im rho^0_01) and the Fermi data (e_l, g_l = df/dT,
//     gp_l = dg/de), rewritten once per temperature;
//   * with D = T^0 - T^1, Y = 1 (x) T^1 + rho1^0 (x) D, where
//     T^{l1} = w_{l1 1} 1 + (w_{l1 0} - w_{l1 1}) rho2^0;  Y is Hermitian in the sense
//     Y[(t3 t1),(t4 t2)] = conj(Y[(t1 t3),(t2 t4)]), so only 4 real and 6 complex
//     entries are formed;
//   * the row sums W[dy] = sum_ky e^{-i ky dy} Y keep, for each complex pair
//     (Z, conj Z), the real sums of c Re Z, s Im Z, c Im Z, s Re Z, which give both
//     members; dy = 0 needs no phase;
//   * the records are stored as three float4 planes transposed to [ky][kx], so the
//     32 columns of a warp read 512 contiguous bytes per plane (coalesced), and each
//     thread loads the next row while it computes the current one; rows advance
//     without integer division.
// One thread per fine-mesh column, one CTA per (transfer momentum, 64 columns, row range).
// The flush and the partial layout are the ones of k_loops.cu, so the same
// deterministic reduction kernel finishes the sum.
#include <cmath>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int MAXD = 9;
constexpr int WARPS = 2;

constexpr int RECF4 = 3;         // float4 planes per record
constexpr int RING = 4;          // rows of records in flight per thread (asynchronous copies into shared memory)

// Shared memory of one CTA: the phase table, then one region per warp that holds the warp's ring of
// record rows during the k-sum ([RING][2 sides x 3 planes][32 lanes] float4) and its flush buffer
// (32 x (2 NDYH 16 + 1) floats) after it.
__host__ __device__ constexpr size_t warp_region_bytes(int ndyh)
{
    return ((sizeof(float) * 32 * (2 * ndyh * 16 + 1) > sizeof(float4) * RING * 2 * RECF4 * 32
                 ? sizeof(float) * 32 * (2 * ndyh * 16 + 1)
                 : sizeof(float4) * RING * 2 * RECF4 * 32) + 15) & ~size_t(15);
}
inline size_t loops2_smem_bytes(int Lf, int ndyh)
{
    return ((sizeof(float2) * Lf + 15) & ~size_t(15)) + WARPS * warp_region_bytes(ndyh);
}

struct Args2 {
    const float4 *rec;       // [3][Lf][Lf] planes, index [j][ky][kx]:
                             //   (rho00, Re rho01, Im rho01, e0), (e1, g0, g1, gp0), (gp1, -, -, -)
    float2 *part;            // [Nq][n_part][ndx][ndyh][16]
    int Lq, nc, Lf, ndx, ndyh;
    int dxs[MAXD], dys[MAXD];
    unsigned needed[MAXD];
    int ky_chunks, ky_len;
    float thr;               // degenerate-pair switch, used when Tp is null
    const double *Tp;        // device flow scale (T, or Lambda with the momentum shell): switch = 1e-2 * T
    float shell_T;           // > 0: momentum-shell regulator at this fixed temperature (records hold f, h)
    const int *s_list;       // optional: CTA x evaluates transfer momentum s_list[x] (partials indexed by x)
    const int *skip;         // optional: the whole launch returns at once when *skip != 0
    const float2 *ptab;      // optional: e^{-2 pi i n / Lf}, n < Lf (computed in the kernel when null)
};

// (t1,t3,t2,t4) -> ab index of the compact loop (P: a=(t2,t1), b=(t4,t3); C: a=(t1,t2), b=(t3,t4))
template <int WHICH>
__host__ __device__ constexpr int abx(int t1, int t3, int t2, int t4)
{
    return WHICH == 0 ? ((t2 * 2 + t1) * 4 + t4 * 2 + t3) : ((t1 * 2 + t2) * 4 + t3 * 2 + t4);
}

template <int WHICH, bool SHELL>
__device__ __forceinline__ float pw(float e1, float g1, float gp1, float e2, float g2, float gp2, float thr, float lam)
{
    if (SHELL) return shell_weight<WHICH, float>(e1, g1, gp1, e2, g2, gp2, thr, lam);   // (g, gp) = (f, h)
    if (WHICH == 0) {
        const float s = e1 + e2;
        return fabsf(s) > thr ? -__fdividef(g1 + g2, s) : -0.5f * (gp1 + gp2);
    } else {
        const float d = e1 - e2;
        return fabsf(d) > thr ? __fdividef(g1 - g2, d) : 0.5f * (gp1 + gp2);
    }
}

// SHELL: momentum-shell regulator (a separate instantiation, so that the temperature flow's code is unchanged)
template <int NDYH, int WHICH, bool SHELL = false>
__global__ void __launch_bounds__(32 * WARPS) loops2_kernel(Args2 a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.skip && *a.skip) return;   // uniform over the grid
    float2 *ptab = reinterpret_cast<float2 *>(smem_raw);
    const int Lf = a.Lf;
    if (a.ptab) {
        for (int n = threadIdx.x; n < Lf; n += blockDim.x) ptab[n] = a.ptab[n];
    } else {
        for (int n = threadIdx.x; n < Lf; n += blockDim.x) {
            double sn, cs;
            sincospi(2.0 * (double)n / (double)Lf, &sn, &cs);
            ptab[n] = make_float2((float)cs, (float)-sn);   // e^{-2 pi i n / Lf}
        }
    }
    __syncthreads();

    constexpr int NT = 32 * WARPS;
    const int s = blockIdx.x;                                    // slot of the partial sums
    const int sq = a.s_list ? a.s_list[blockIdx.x] : blockIdx.x;  // transfer momentum
    const int sx = (sq / a.Lq) * a.nc, sy = (sq % a.Lq) * a.nc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *region = smem_raw + ((sizeof(float2) * Lf + 15) & ~size_t(15)) + warp * warp_region_bytes(NDYH);
    float4 *ring = reinterpret_cast<float4 *>(region);   // [RING][6][32]: rows in flight of this warp's columns
    const int kx = blockIdx.y * NT + threadIdx.x;
    // temperature flow: the scale is T; momentum shell: the scale is Lambda and the temperature is fixed
    const float lam = SHELL ? (float)*a.Tp : 0.f;
    const float thr = SHELL ? 1e-2f * a.shell_T : (a.Tp ? (float)(1e-2 * *a.Tp) : a.thr);
    const bool valid = kx < Lf;
    const int kyc = blockIdx.z;
    const int ky0 = kyc * a.ky_len;
    const int ky1 = min(Lf, ky0 + a.ky_len);

    float R0[4], P0y[6], P0z[6];
    float Rc[NDYH > 1 ? NDYH - 1 : 1][4], Rs[NDYH > 1 ? NDYH - 1 : 1][4];
    float Pcy[NDYH > 1 ? NDYH - 1 : 1][6], Psz[NDYH > 1 ? NDYH - 1 : 1][6];
    float Pcz[NDYH > 1 ? NDYH - 1 : 1][6], Psy[NDYH > 1 ? NDYH - 1 : 1][6];
#pragma unroll
    for (int j = 0; j < 4; j++) R0[j] = 0.f;
#pragma unroll
    for (int j = 0; j < 6; j++) { P0y[j] = 0.f; P0z[j] = 0.f; }
#pragma unroll
    for (int i = 0; i < NDYH - 1; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++) { Rc[i][j] = 0.f; Rs[i][j] = 0.f; }
#pragma unroll
        for (int j = 0; j < 6; j++) { Pcy[i][j] = 0.f; Psz[i][j] = 0.f; Pcz[i][j] = 0.f; Psy[i][j] = 0.f; }
    }

    if (valid && ky0 < ky1) {
        // columns of k1 and k2; rows step by +1 on the q side and by -1 on the s - q side
        const int k1x = WHICH == 0 ? (sx - kx + Lf) % Lf : kx;
        const int k2x = WHICH == 0 ? kx : (kx - sx + Lf) % Lf;
        int k1y = WHICH == 0 ? ((sy - ky0) % Lf + Lf) % Lf : ky0;
        int k2y = WHICH == 0 ? ky0 : ((ky0 - sy) % Lf + Lf) % Lf;
        const size_t plane = (size_t)Lf * Lf;
        int o1 = k1y * Lf + k1x, o2 = k2y * Lf + k2x;        // offsets of the next row to be copied
        const int wrap = (Lf - 1) * Lf;
        // copy one row (both sides, three planes) into ring slot sl, then step the offsets to the next
        // row: the q side moves by +Lf, the s - q side by -Lf (P), both +Lf (C), with wrap
        auto issue_row = [&](int sl) {
            float4 *r = ring + sl * 2 * RECF4 * 32 + lane;
#pragma unroll
            for (int pl = 0; pl < RECF4; pl++) {
                cp_async16(r + pl * 32, a.rec + pl * plane + o1);
                cp_async16(r + (RECF4 + pl) * 32, a.rec + pl * plane + o2);
            }
            if (WHICH == 0) { o1 = o1 >= Lf ? o1 - Lf : o1 + wrap; o2 = o2 < wrap ? o2 + Lf : o2 - wrap; }
            else            { o1 = o1 < wrap ? o1 + Lf : o1 - wrap; o2 = o2 < wrap ? o2 + Lf : o2 - wrap; }
        };
#pragma unroll
        for (int i = 0; i < RING - 1; i++) {   // rows ky0 .. ky0 + RING - 2 in flight
            if (ky0 + i < ky1) issue_row(i);
            cp_async_commit();
        }
        int pn[MAXD];
#pragma unroll
        for (int i = 1; i < NDYH; i++) pn[i] = (int)(((long)ky0 * a.dys[i]) % Lf);
        const float sgn = WHICH == 0 ? 1.f : -1.f;
        for (int ky = ky0; ky < ky1; ky++) {
            const int it = ky - ky0;
            if (ky + RING - 1 < ky1) issue_row((it + RING - 1) & (RING - 1));
            cp_async_commit();
            cp_async_wait<RING - 1>();   // this thread's copies of row ky have landed
            const float4 *r = ring + (it & (RING - 1)) * 2 * RECF4 * 32 + lane;
            const float4 a0 = r[0], a1 = r[32], a2 = r[64], b0 = r[96], b1 = r[128], b2 = r[160];
            // pair weights w[l1][l2]: l1 on k1, l2 on k2
            const float e1[2] = {a0.w, a1.x}, g1[2] = {a1.y, a1.z}, gp1[2] = {a1.w, a2.x};
            const float e2[2] = {b0.w, b1.x}, g2[2] = {b1.y, b1.z}, gp2[2] = {b1.w, b2.x};
            float w[2][2];
#pragma unroll
            for (int l1 = 0; l1 < 2; l1++)
#pragma unroll
                for (int l2 = 0; l2 < 2; l2++) w[l1][l2] = pw<WHICH, SHELL>(e1[l1], g1[l1], gp1[l1], e2[l2], g2[l2], gp2[l2], thr, lam);
            // T^{l1} = w_{l1 1} 1 + (w_{l1 0} - w_{l1 1}) rho2'^0 ;  D = T^0 - T^1
            const float A2 = b0.x, C2r = b0.y, C2i = sgn * b0.z;    // rho2' = rho2 (P) or conj(rho2) (C)
            const float dw0 = w[0][0] - w[0][1], dw1 = w[1][0] - w[1][1];
            const float T1_00 = fmaf(dw1, A2, w[1][1]), T1_11 = fmaf(dw1, 1.f - A2, w[1][1]);
            const float T1r = dw1 * C2r, T1i = dw1 * C2i;
            const float dd = dw0 - dw1, dd0 = w[0][1] - w[1][1];
            const float D00 = fmaf(dd, A2, dd0), D11 = fmaf(dd, 1.f - A2, dd0);
            const float Dr = dd * C2r, Di = dd * C2i;
            // Y = 1 (x) T^1 + rho1^0 (x) D: 4 real and 6 complex independent entries
            const float A1 = a0.x, B1 = 1.f - a0.x, C1r = a0.y, C1i = a0.z;
            float X[4], Zy[6], Zz[6];
            X[0] = fmaf(A1, D00, T1_00);    // Y[00][00]
            X[1] = fmaf(A1, D11, T1_11);    // Y[00][11]
            X[2] = fmaf(B1, D00, T1_00);    // Y[11][00]
            X[3] = fmaf(B1, D11, T1_11);    // Y[11][11]
            Zy[0] = fmaf(A1, Dr, T1r); Zz[0] = fmaf(A1, Di, T1i);   // Y[00][01]
            Zy[1] = fmaf(B1, Dr, T1r); Zz[1] = fmaf(B1, Di, T1i);   // Y[11][01]
            Zy[2] = C1r * D00; Zz[2] = C1i * D00;                   // Y[01][00]
            Zy[3] = C1r * D11; Zz[3] = C1i * D11;                   // Y[01][11]
            Zy[4] = C1r * Dr - C1i * Di; Zz[4] = C1r * Di + C1i * Dr;   // Y[01][01] = rho01 D01
            Zy[5] = C1r * Dr + C1i * Di; Zz[5] = C1i * Dr - C1r * Di;   // Y[01][10] = rho01 conj(D01)
            // row sums
#pragma unroll
            for (int j = 0; j < 4; j++) R0[j] += X[j];
#pragma unroll
            for (int j = 0; j < 6; j++) { P0y[j] += Zy[j]; P0z[j] += Zz[j]; }
#pragma unroll
            for (int i = 1; i < NDYH; i++) {
                const float2 ph = ptab[pn[i]];
                pn[i] += a.dys[i];
                if (pn[i] >= Lf) pn[i] -= Lf;
#pragma unroll
                for (int j = 0; j < 4; j++) { Rc[i - 1][j] = fmaf(ph.x, X[j], Rc[i - 1][j]); Rs[i - 1][j] = fmaf(ph.y, X[j], Rs[i - 1][j]); }
#pragma unroll
                for (int j = 0; j < 6; j++) {
                    Pcy[i - 1][j] = fmaf(ph.x, Zy[j], Pcy[i - 1][j]);
                    Psz[i - 1][j] = fmaf(ph.y, Zz[j], Psz[i - 1][j]);
                    Pcz[i - 1][j] = fmaf(ph.x, Zz[j], Pcz[i - 1][j]);
                    Psy[i - 1][j] = fmaf(ph.y, Zy[j], Psy[i - 1][j]);
                }
            }
        }
        cp_async_wait<0>();   // nothing in flight before the region is reused below (trailing groups are empty)
    }

    // ---- rebuild W[dy][ab] from the paired sums
    constexpr int XR[4] = {abx<WHICH>(0, 0, 0, 0), abx<WHICH>(0, 0, 1, 1), abx<WHICH>(1, 1, 0, 0), abx<WHICH>(1, 1, 1, 1)};
    constexpr int ZA[6] = {abx<WHICH>(0, 0, 0, 1), abx<WHICH>(1, 1, 0, 1), abx<WHICH>(0, 1, 0, 0),
                           abx<WHICH>(0, 1, 1, 1), abx<WHICH>(0, 1, 0, 1), abx<WHICH>(0, 1, 1, 0)};
    constexpr int ZB[6] = {abx<WHICH>(0, 0, 1, 0), abx<WHICH>(1, 1, 1, 0), abx<WHICH>(1, 0, 0, 0),
                           abx<WHICH>(1, 0, 1, 1), abx<WHICH>(1, 0, 1, 0), abx<WHICH>(1, 0, 0, 1)};
    float2 W[NDYH][16];
#pragma unroll
    for (int j = 0; j < 4; j++) W[0][XR[j]] = make_float2(R0[j], 0.f);
#pragma unroll
    for (int j = 0; j < 6; j++) {
        W[0][ZA[j]] = make_float2(P0y[j], P0z[j]);
        W[0][ZB[j]] = make_float2(P0y[j], -P0z[j]);
    }
#pragma unroll
    for (int i = 1; i < NDYH; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++) W[i][XR[j]] = make_float2(Rc[i - 1][j], Rs[i - 1][j]);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            W[i][ZA[j]] = make_float2(Pcy[i - 1][j] - Psz[i - 1][j], Pcz[i - 1][j] + Psy[i - 1][j]);
            W[i][ZB[j]] = make_float2(Pcy[i - 1][j] + Psz[i - 1][j], Psy[i - 1][j] - Pcz[i - 1][j]);
        }
    }

    // ---- flush: per distinct dx, multiply by e^{-i kx dx}, sum the warp through smem
    constexpr int NV = 2 * NDYH * 16;
    constexpr int PITCH = NV + 1;
    float *buf = reinterpret_cast<float *>(region);
    __syncwarp();   // every lane of the warp is done with its ring entries (lanes past Lf skipped the k-sum)
    const int n_part = gridDim.y * WARPS * gridDim.z;
    const int p = (blockIdx.y * WARPS + warp) * gridDim.z + kyc;
    for (int dxi = 0; dxi < a.ndx; dxi++) {
        if (a.needed[dxi] == 0) continue;
        const int n = (int)((((long)kx * a.dxs[dxi]) % Lf + Lf) % Lf);
        const float2 phx = valid ? ptab[n] : make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < NDYH; i++)
#pragma unroll
            for (int j = 0; j < 16; j++) {
                buf[lane * PITCH + 2 * (i * 16 + j)] = phx.x * W[i][j].x - phx.y * W[i][j].y;
                buf[lane * PITCH + 2 * (i * 16 + j) + 1] = phx.x * W[i][j].y + phx.y * W[i][j].x;
            }
        __syncwarp();
        for (int v = lane; v < NV; v += 32) {
            float acc = 0.f;
#pragma unroll 8
            for (int r = 0; r < 32; r++) acc += buf[r * PITCH + v];
            const int i = v / 32, j = (v / 2) % 16, re = v & 1;
            if ((a.needed[dxi] >> i) & 1u) {
                const size_t o = ((((size_t)s * n_part + p) * a.ndx + dxi) * a.ndyh + i) * 16 + j;
                reinterpret_cast<float *>(a.part)[2 * o + re] = acc;
            }
        }
        __syncwarp();
    }
}

// Record of one fine k (FP32, three planes [j][ky][kx]): plane 0 = (rho00, Re rho01, Im rho01, e0),
// plane 1 = (e1, g0, g1, g'0), plane 2 = (g'1, 0, 0, 0), with e = E - mu, g = dF/dT-type weight
// derivative of the Fermi function and g' its derivative in e.  The projector and e do not depend on
// T and are written once per model; only g and g' are refreshed per evaluation.
__global__ void rec_static_kernel(const double *E, const double2 *U, int Nk, int Lf, double mu, float4 *rec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nk) return;
    // rho^0 = U_{.0} U*_{.0}: rho00 = |U_00|^2, rho01 = U_00 conj(U_10)
    const double2 u0 = U[(size_t)k * 4 + 0], u1 = U[(size_t)k * 4 + 2];
    const int kx = k / Lf, ky = k % Lf;
    const size_t t = (size_t)ky * Lf + kx, plane = (size_t)Lf * Lf;
    rec[t] = make_float4((float)(u0.x * u0.x + u0.y * u0.y), (float)(u0.x * u1.x + u0.y * u1.y),
                         (float)(u0.y * u1.x - u0.x * u1.y), (float)(E[2 * k] - mu));
    rec[plane + t] = make_float4((float)(E[2 * k + 1] - mu), 0.f, 0.f, 0.f);
    rec[2 * plane + t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// g = -df/dT = (x / T) f (1 - f) and g' = dg/de with x = e / T, in the overflow-safe form with
// z = exp(-|x|): f (1 - f) = z / (1 + z)^2 and dg/de = f (1 - f) / T^2 (1 - |x| (1 - z) / (1 + z)).
// FP32 (the split path's loop sums are FP32).
__global__ void rec_T_kernel(int n, double T_value, const double *Tp, float4 *rec)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float invT = 1.f / (float)(Tp ? *Tp : T_value);   // device-resident temperature when given
    const float e[2] = {rec[t].w, rec[n + t].x};
    float g[2], gp[2];
#pragma unroll
    for (int l = 0; l < 2; l++) {
        const float x = e[l] * invT, ax = fabsf(x);
        const float z = expf(-ax), opz = 1.f + z;
        const float h = z / (opz * opz);
        g[l] = x * invT * h;
        gp[l] = h * invT * invT * (1.f - ax * (1.f - z) / opz);
    }
    rec[n + t] = make_float4(e[1], g[0], g[1], gp[0]);
    rec[2 * n + t] = make_float4(gp[1], 0.f, 0.f, 0.f);
}

// Momentum-shell records: (f, h) = (f(e), f (1 - f) / T) at the fixed temperature T in the slots of
// (g, g'), from the FP64 energies (written once per model; the shell weight needs no T-dependent data).
__global__ void rec_shell_kernel(const double *E, int Nk, int Lf, double mu, double T, float4 *rec)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nk) return;
    const int kx = k / Lf, ky = k % Lf;
    const size_t t = (size_t)ky * Lf + kx, plane = (size_t)Lf * Lf;
    double f[2], h[2];
    for (int l = 0; l < 2; l++) {
        const double e = E[2 * k + l] - mu, z = exp(-fabs(e) / T);
        f[l] = e > 0 ? z / (1.0 + z) : 1.0 / (1.0 + z);
        h[l] = z / ((1.0 + z) * (1.0 + z)) / T;
    }
    const float e1 = rec[plane + t].x;
    rec[plane + t] = make_float4(e1, (float)f[0], (float)f[1], (float)h[0]);
    rec[2 * plane + t] = make_float4((float)h[1], 0.f, 0.f, 0.f);
}

template <int NDYH, int WHICH>
cudaError_t launch2(tufrg_model *m, const Args2 &a, int n_s)
{
    dim3 grid(n_s, (m->Lf + 32 * WARPS - 1) / (32 * WARPS), a.ky_chunks);
    const size_t smem = loops2_smem_bytes(m->Lf, NDYH);
    auto kern = a.shell_T > 0.f ? loops2_kernel<NDYH, WHICH, true> : loops2_kernel<NDYH, WHICH, false>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhaseScope ps(m, PH_LOOPS);
    kern<<<grid, 32 * WARPS, smem, m->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

// Resident CTAs per SM of the instantiation this model launches (occupancy API).
int loops2_blocks_per_sm(const tufrg_model *m)
{
    int ndyh = 0;
    for (int v : m->dys) ndyh += v >= 0;
    const size_t smem = loops2_smem_bytes(m->Lf, ndyh);
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (ndyh == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, loops2_kernel<1, 0>, 32 * WARPS, smem);
    if (ndyh == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, loops2_kernel<2, 0>, 32 * WARPS, smem);
    if (ndyh == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, loops2_kernel<3, 0>, 32 * WARPS, smem);
    if (ndyh == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, loops2_kernel<4, 0>, 32 * WARPS, smem);
    if (ndyh == 5) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, loops2_kernel<5, 0>, 32 * WARPS, smem);
    return (e == cudaSuccess && n > 0) ? n : 4;
}

bool loops2_supported(const tufrg_model *m)
{
    int ndyh = 0;
    for (int v : m->dys) ndyh += v >= 0;
    return m->ns == 2 && m->precision != TUFRG_FP64 && ndyh <= 5 && (int)m->dxs.size() <= MAXD;
}

cudaError_t launch_loop_records_static(tufrg_model *m)
{
    rec_static_kernel<<<(m->Nk + 255) / 256, 256, 0, m->stream>>>(m->d_E, m->d_U, m->Nk, m->Lf, m->mu, m->d_rec);
    return cudaGetLastError();
}

cudaError_t launch_loop_records_shell(tufrg_model *m)
{
    rec_shell_kernel<<<(m->Nk + 255) / 256, 256, 0, m->stream>>>(m->d_E, m->Nk, m->Lf, m->mu, m->T_reg, m->d_rec);
    return cudaGetLastError();
}

cudaError_t launch_loop_records(tufrg_model *m)
{
    if (m->regulator == TUFRG_REG_MOMENTUM_SHELL) return cudaSuccess;   // the shell records do not depend on Lambda
    PhaseScope ps(m, PH_FERMI);
    rec_T_kernel<<<(m->Nk + 255) / 256, 256, 0, m->stream>>>(m->Nk, 0.0, m->d_scal, m->d_rec);
    return cudaGetLastError();
}

// Loop sums of channel ch into the partial buffer (no reduction).  With s_list, only the
// listed transfer momenta (n_list of them) are evaluated, into partial slots 0..n_list-1 of part.
cudaError_t launch_loops2_ex(tufrg_model *m, int ch, const int *s_list, int n_list, float2 *part, const int *skip)
{
    const LoopPlan &pl = m->plan;
    Args2 a{};
    a.rec = m->d_rec;
    a.part = part;
    a.s_list = s_list;
    a.skip = skip;
    a.Lq = m->Lq; a.nc = m->nc; a.Lf = m->Lf;
    a.ndx = (int)m->dxs.size();
    int ndyh = 0;
    for (int v : m->dys)
        if (v >= 0) a.dys[ndyh++] = v;
    a.ndyh = ndyh;
    for (int i = 0; i < a.ndx; i++) {
        a.dxs[i] = m->dxs[i];
        a.needed[i] = 0;
        for (int j = 0; j < ndyh; j++) {
            const int dx = m->dxs[i], dy = a.dys[j];
            bool in = false;
            for (int d = 0; d < m->nd; d++) in |= (m->deltas[2 * d] == dx && m->deltas[2 * d + 1] == dy);
            if (in && (dy > 0 || dx >= 0)) a.needed[i] |= 1u << j;
        }
    }
    a.ky_chunks = pl.ky_chunks;
    a.ky_len = (m->Lf + pl.ky_chunks - 1) / pl.ky_chunks;
    a.thr = 0.f;
    a.Tp = m->d_scal;
    a.shell_T = m->regulator == TUFRG_REG_MOMENTUM_SHELL ? (float)m->T_reg : 0.f;
    a.ptab = m->d_lph32;
    const int n_s = s_list ? n_list : m->Nq;
    switch (ndyh) {
    case 1: return ch == 0 ? launch2<1, 0>(m, a, n_s) : launch2<1, 1>(m, a, n_s);
    case 2: return ch == 0 ? launch2<2, 0>(m, a, n_s) : launch2<2, 1>(m, a, n_s);
    case 3: return ch == 0 ? launch2<3, 0>(m, a, n_s) : launch2<3, 1>(m, a, n_s);
    case 4: return ch == 0 ? launch2<4, 0>(m, a, n_s) : launch2<4, 1>(m, a, n_s);
    case 5: return ch == 0 ? launch2<5, 0>(m, a, n_s) : launch2<5, 1>(m, a, n_s);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_loops2(tufrg_model *m, int ch)
{
    // with loop symmetries only the orbit representatives are summed (partial slots = list positions)
    return launch_loops2_ex(m, ch, m->sym ? m->d_loop_list : nullptr, m->sym ? m->n_loop_q : 0,
                            reinterpret_cast<float2 *>(m->d_part), m->sur ? m->d_sur_flag : nullptr);
}

}  // namespace tufrg

// ---------------------------------------------------------------------------------
// Loop k-sum without allocation: the same kernels with their scratch in a static array.
// ---------------------------------------------------------------------------------
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

namespace tufrg {
namespace {

// Records of one fine mesh plus the partial sums of one channel; see tufrg.h.
__device__ __align__(256) unsigned char g_noalloc_scratch[TUFRG_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAXND = 64;
constexpr int NOALLOC_MAXDEV = 64;

struct NoallocTables {
    int nd;
    int d[2 * NOALLOC_MAXND];      // sorted bond differences (dx, dy)
    int slot[NOALLOC_MAXND];       // dxi * ndyh + dyi of the half-plane representative
};

// Fixed-order sum of the partials, scaled by 1/Nk; writes both Hermitian halves (FP64).
__global__ void noalloc_reduce_kernel(const float2 *part, int n_part, int ndx, int ndyh, NoallocTables t, int Nq,
                                      double inv_nk, double2 *out)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)Nq * t.nd * 16) return;
    const int ab = idx % 16;
    const int d = (idx / 16) % t.nd;
    const int s = (int)(idx / (16 * (size_t)t.nd));
    const int dx = t.d[2 * d], dy = t.d[2 * d + 1];
    const bool half = dy > 0 || (dy == 0 && dx >= 0);
    const int src_ab = half ? ab : (ab % 4) * 4 + ab / 4;
    double re = 0.0, im = 0.0;
    for (int p = 0; p < n_part; p++) {
        const float2 v = part[(((size_t)s * n_part + p) * ndx * ndyh + t.slot[d]) * 16 + src_ab];
        re += (double)v.x;
        im += (double)v.y;
    }
    out[idx] = make_double2(re * inv_nk, (half ? im : -im) * inv_nk);
}

std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAXDEV] = {};

}  // namespace
}  // namespace tufrg

extern "C" tufrg_status tufrg_loops_noalloc(int Lq, int nc, const double *d_E, const double *d_U, double mu, double T,
                                            int n_ff, const int *h_ffR, int channel_mask, void *d_loops,
                                            void *cuda_stream)
{
    using namespace tufrg;
    if (Lq < 2 || nc < 1 || (long)Lq * nc > 4096 || !d_E || !d_U || !h_ffR || !d_loops || n_ff < 1)
        return TUFRG_EINVAL;
    if (!(T > 0) || !std::isfinite(T) || !std::isfinite(mu) || (channel_mask & ~3)) return TUFRG_EINVAL;
    if (h_ffR[0] != 0 || h_ffR[1] != 0) return TUFRG_EINVAL;
    const int Lf = Lq * nc;
    const size_t Nk = (size_t)Lf * Lf;
    const int Nq = Lq * Lq;
    // bond differences (sorted) and their separable parts, as the model builds them
    std::vector<std::pair<int, int>> dl;
    for (int i = 0; i < n_ff; i++)
        for (int j = 0; j < n_ff; j++) dl.emplace_back(h_ffR[2 * i] - h_ffR[2 * j], h_ffR[2 * i + 1] - h_ffR[2 * j + 1]);
    std::sort(dl.begin(), dl.end());
    dl.erase(std::unique(dl.begin(), dl.end()), dl.end());
    std::vector<int> xs, ys;
    for (auto &p : dl) { xs.push_back(p.first); ys.push_back(p.second); }
    std::sort(xs.begin(), xs.end()); xs.erase(std::unique(xs.begin(), xs.end()), xs.end());
    std::sort(ys.begin(), ys.end()); ys.erase(std::unique(ys.begin(), ys.end()), ys.end());
    std::vector<int> dyh;
    for (int v : ys) if (v >= 0) dyh.push_back(v);
    const int ndx = (int)xs.size(), ndyh = (int)dyh.size(), nd = (int)dl.size();
    if (ndyh < 1 || ndyh > 3 || ndx > MAXD || nd > NOALLOC_MAXND) return TUFRG_ENOTSUP;
    // scratch budget: records, then the partials of one channel (one row range per column)
    const int ctas_x = (Lf + 32 * WARPS - 1) / (32 * WARPS);
    const int n_part = ctas_x * WARPS;
    const size_t rec_bytes = ((Nk * RECF4 * sizeof(float4)) + 255) & ~size_t(255);
    const size_t part_bytes = (size_t)Nq * n_part * ndx * ndyh * 16 * sizeof(float2);
    if (rec_bytes + part_bytes > (size_t)TUFRG_NOALLOC_SCRATCH_BYTES) return TUFRG_ETOOBIG;
    // device address of the static scratch (the device must be current).  Outside stream capture it is looked
    // up on every call, so that a device reset or a new primary context never leaves a stale address behind;
    // during capture the address of the last uncaptured call on this device is used.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAXDEV) return TUFRG_ECUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
    if (capturing) (void)cudaGetLastError();   // clear the (non-sticky) error a refused capture query leaves
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!capturing) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TUFRG_ECUDA;
            g_noalloc_addr[dev] = p;
        }
        base = g_noalloc_addr[dev];
    }
    if (!base) return TUFRG_ECUDA;   // first call on this device inside a capture: nothing looked up yet
    float4 *rec = reinterpret_cast<float4 *>(base);
    float2 *part = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(base) + rec_bytes);

    rec_static_kernel<<<(unsigned)((Nk + 255) / 256), 256, 0, st>>>(d_E, reinterpret_cast<const double2 *>(d_U), (int)Nk,
                                                                      Lf, mu, rec);
    rec_T_kernel<<<(unsigned)((Nk + 255) / 256), 256, 0, st>>>((int)Nk, T, nullptr, rec);
    if (cudaGetLastError() != cudaSuccess) return TUFRG_ECUDA;
    Args2 a{};
    a.rec = rec;
    a.part = part;
    a.Lq = Lq; a.nc = nc; a.Lf = Lf; a.ndx = ndx; a.ndyh = ndyh;
    for (int j = 0; j < ndyh; j++) a.dys[j] = dyh[j];
    for (int i = 0; i < ndx; i++) {
        a.dxs[i] = xs[i];
        a.needed[i] = 0;
        for (int j = 0; j < ndyh; j++) {
            const bool in = std::binary_search(dl.begin(), dl.end(), std::make_pair(xs[i], dyh[j]));
            if (in && (dyh[j] > 0 || xs[i] >= 0)) a.needed[i] |= 1u << j;
        }
    }
    a.ky_chunks = 1;
    a.ky_len = Lf;
    a.thr = (float)(1e-2 * T);
    a.Tp = nullptr;
    NoallocTables t{};
    t.nd = nd;
    for (int k = 0; k < nd; k++) {
        int dx = dl[k].first, dy = dl[k].second;
        t.d[2 * k] = dx;
        t.d[2 * k + 1] = dy;
        if (!(dy > 0 || (dy == 0 && dx >= 0))) { dx = -dx; dy = -dy; }
        const int xi = (int)(std::find(xs.begin(), xs.end(), dx) - xs.begin());
        const int yi = (int)(std::find(dyh.begin(), dyh.end(), dy) - dyh.begin());
        t.slot[k] = xi * ndyh + yi;
    }
    const size_t smem = loops2_smem_bytes(Lf, ndyh);
    const dim3 grid(Nq, ctas_x, 1);
    const size_t per = (size_t)Nq * nd * 16;
    for (int ch = 0; ch < 2; ch++) {
        if (!((channel_mask >> ch) & 1)) continue;
        void (*kern)(Args2) = nullptr;
        if (ndyh == 1) kern = ch == 0 ? loops2_kernel<1, 0> : loops2_kernel<1, 1>;
        if (ndyh == 2) kern = ch == 0 ? loops2_kernel<2, 0> : loops2_kernel<2, 1>;
        if (ndyh == 3) kern = ch == 0 ? loops2_kernel<3, 0> : loops2_kernel<3, 1>;
        if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return TUFRG_ECUDA;
        kern<<<grid, 32 * WARPS, smem, st>>>(a);
        if (cudaGetLastError() != cudaSuccess) return TUFRG_ECUDA;
        noalloc_reduce_kernel<<<(unsigned)((per + 255) / 256), 256, 0, st>>>(
            part, n_part, ndx, ndyh, t, Nq, 1.0 / (double)Nk, reinterpret_cast<double2 *>(d_loops) + ch * per);
        if (cudaGetLastError() != cudaSuccess) return TUFRG_ECUDA;
    }
    return TUFRG_OK;
}
