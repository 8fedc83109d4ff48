// Form factors of the irreducible representations of C4v (Sec. 2: orthonormal linear combinations of the plane
// waves f_R(k) = e^{-ik.R} that transform under an irreducible representation of the point group).
//
// For a bond set closed under the eight point operations of the square lattice, the bonds fall into shells (orbits
// of the group).  On each shell the permutation representation D(g) is projected with the characters of A1, A2,
// B1, B2 and E, P = (d / 8) sum_g chi(g) D(g), and the images of the shell's unit vectors are orthonormalised
// (modified Gram-Schmidt), giving real rows W[i][R] with f_i(k) = sum_R W[i][R] f_R(k).  W is orthogonal, so the
// exchange propagators in that basis are X' = (W x 1) X (W x 1)^T per transfer momentum and channel (1 on the
// orbital pairs): the same flow written in other form factors.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

// the point operations (integer matrices on (x, y)) and their class: 0 identity, 1 quarter turns, 2 half turn,
// 3 axis mirrors, 4 diagonal mirrors; characters [irrep][class] of A1, A2, B1, B2, E
constexpr int OPS[8][5] = {{1, 0, 0, 1, 0}, {0, -1, 1, 0, 1}, {0, 1, -1, 0, 1}, {-1, 0, 0, -1, 2},
                           {1, 0, 0, -1, 3}, {-1, 0, 0, 1, 3}, {0, 1, 1, 0, 4}, {0, -1, -1, 0, 4}};
constexpr int CHI[5][5] = {{1, 1, 1, 1, 1}, {1, 1, 1, -1, -1}, {1, -1, 1, 1, -1}, {1, -1, 1, -1, 1}, {2, 0, -2, 0, 0}};
constexpr int DIM[5] = {1, 1, 1, 1, 2};

// out[c][q][(i,a)][(j,b)] = sum_{R,R'} W[i][R] W[j][R'] X[c][q][(R,a)][(R',b)]  (inverse: W^T for W)
__global__ void irrep_kernel(const double2 *X, int Nq, int nff, int ns2, const double *Wg, int inverse, double2 *out)
{
    extern __shared__ double Ws[];   // [nff][nff], rows = target form factors
    for (int t = threadIdx.x; t < nff * nff; t += blockDim.x) {
        const int i = t / nff, r = t % nff;
        Ws[t] = inverse ? Wg[r * nff + i] : Wg[t];
    }
    __syncthreads();
    const int M = nff * ns2;
    const size_t M2 = (size_t)M * M;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t cq = blockIdx.y;   // channel * Nq + q
    if (e >= M2) return;
    const int row = (int)(e / M), col = (int)(e % M);
    const int i = row / ns2, a = row % ns2, j = col / ns2, b = col % ns2;
    const double2 *Xq = X + cq * M2;
    double re = 0.0, im = 0.0;
    for (int r = 0; r < nff; r++) {
        const double wi = Ws[i * nff + r];
        if (wi == 0.0) continue;
        double sr = 0.0, si = 0.0;
        for (int rp = 0; rp < nff; rp++) {
            const double wj = Ws[j * nff + rp];
            if (wj == 0.0) continue;
            const double2 x = Xq[((size_t)(r * ns2 + a)) * M + rp * ns2 + b];
            sr = fma(wj, x.x, sr);
            si = fma(wj, x.y, si);
        }
        re = fma(wi, sr, re);
        im = fma(wi, si, im);
    }
    out[cq * M2 + e] = make_double2(re, im);
}

}  // namespace

// Builds the irrep basis of the model's bond set (host); false when the set is not closed under C4v.
bool build_irrep_basis(tufrg_model *m)
{
    const int n = m->nff;
    std::map<std::pair<int, int>, int> idx;
    for (int i = 0; i < n; i++) idx[{m->ffR[2 * i], m->ffR[2 * i + 1]}] = i;
    auto act = [&](int g, int i) {   // index of g R_i, or -1
        const int x = m->ffR[2 * i], y = m->ffR[2 * i + 1];
        auto it = idx.find({OPS[g][0] * x + OPS[g][1] * y, OPS[g][2] * x + OPS[g][3] * y});
        return it == idx.end() ? -1 : it->second;
    };
    for (int i = 0; i < n; i++)
        for (int g = 0; g < 8; g++)
            if (act(g, i) < 0) return false;
    std::vector<int> shell(n, -1);
    int nshell = 0;
    std::vector<double> W;
    std::vector<int> lab;
    for (int i0 = 0; i0 < n; i0++) {
        if (shell[i0] >= 0) continue;
        std::vector<int> mem;
        for (int g = 0; g < 8; g++) {
            const int j = act(g, i0);
            if (std::find(mem.begin(), mem.end(), j) == mem.end()) mem.push_back(j);
        }
        std::sort(mem.begin(), mem.end());
        for (int j : mem) shell[j] = nshell;
        for (int gi = 0; gi < 5; gi++) {
            std::vector<std::vector<double>> basis;
            for (int j : mem) {
                // P e_j = (d/8) sum_g chi(g) D(g) e_j, D(g) e_j = e_{g R_j}
                std::vector<double> v(n, 0.0);
                for (int g = 0; g < 8; g++) v[act(g, j)] += DIM[gi] * CHI[gi][OPS[g][4]] / 8.0;
                for (const auto &b : basis) {   // modified Gram-Schmidt against the vectors kept so far
                    double d = 0.0;
                    for (int k = 0; k < n; k++) d += b[k] * v[k];
                    for (int k = 0; k < n; k++) v[k] -= d * b[k];
                }
                double nv = 0.0;
                for (double x : v) nv += x * x;
                nv = std::sqrt(nv);
                if (nv < 1e-9) continue;
                for (double &x : v) x /= nv;
                basis.push_back(v);
            }
            for (size_t p = 0; p < basis.size(); p++) {
                W.insert(W.end(), basis[p].begin(), basis[p].end());
                lab.push_back(nshell);
                lab.push_back(gi);
                lab.push_back((int)p);
            }
        }
        nshell++;
    }
    if ((int)lab.size() != 3 * n) return false;
    m->ffW = W;
    m->ff_labels = lab;
    return true;
}

cudaError_t launch_irrep_basis(tufrg_model *m, const double2 *d_state, int inverse, double2 *d_out)
{
    if (!m->d_ffW) {
        TUFRG_CUDA_TRY(cudaMalloc(&m->d_ffW, sizeof(double) * m->ffW.size()));
        TUFRG_CUDA_TRY(cudaMemcpyAsync(m->d_ffW, m->ffW.data(), sizeof(double) * m->ffW.size(), cudaMemcpyHostToDevice,
                                       m->stream));
    }
    const size_t M2 = (size_t)m->M * m->M;
    const dim3 grid((unsigned)((M2 + 255) / 256), 2 * m->Nq);
    m->launches++;
    irrep_kernel<<<grid, 256, sizeof(double) * m->nff * m->nff, m->stream>>>(d_state, m->Nq, m->nff, m->ns * m->ns,
                                                                           m->d_ffW, inverse, d_out);
    return cudaGetLastError();
}

}  // namespace tufrg
