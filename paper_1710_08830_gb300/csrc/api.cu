// C ABI of libtufrg: model set-up (tables, memory), the right-hand side and the flow.
// Every entry point returns a tufrg_status and never throws across the boundary.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <climits>
#include <array>
#include <complex>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "tufrg_internal.cuh"

using namespace tufrg;

namespace {

int imod(int a, int m)
{
    int r = a % m;
    return r < 0 ? r + m : r;
}

tufrg_status fail(tufrg_model *m, tufrg_status st, const std::string &msg)
{
    if (m) m->err = msg;
    return st;
}

tufrg_status cuda_fail(tufrg_model *m, cudaError_t e, const char *where)
{
    if (m) m->err = std::string(where) + ": " + cudaGetErrorString(e);
    // consume the error: a failed allocation or launch must not stay pending for the caller's next launch check
    // (nor for the next one of this library); a sticky error stays in the context regardless
    (void)cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return TUFRG_ENOMEM;
    return e == cudaErrorNotSupported ? TUFRG_ENOTSUP : TUFRG_ECUDA;
}

// A host allocation that failed inside an entry point (std::bad_alloc, or std::length_error for a size beyond what
// a container holds) is reported as TUFRG_ENOMEM instead of crossing the C boundary.
tufrg_status host_alloc_fail(tufrg_model *m, const std::exception &ex) noexcept
{
    if (m) {
        try {
            m->err = std::string("host allocation failed: ") + ex.what();
        } catch (...) {
            m->err.clear();
        }
    }
    return TUFRG_ENOMEM;
}

#define CK(expr, where)                                        \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return cuda_fail(m, _e, where); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * count);
}

template <typename T>
cudaError_t upload(T **p, const std::vector<T> &v, cudaStream_t s)
{
    cudaError_t e = dalloc(p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    e = cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);   // the host vector may go away
}

int ff_index_mod(const tufrg_model *m, int x, int y)
{
    for (int i = 0; i < m->nff; i++)
        if (imod(m->ffR[2 * i] - x, m->Lq) == 0 && imod(m->ffR[2 * i + 1] - y, m->Lq) == 0) return i;
    return -1;
}

// Bond bookkeeping for the loops: sorted differences, separable dx / dy sets, slots.
void build_loop_tables(tufrg_model *m)
{
    std::vector<std::pair<int, int>> d;
    for (int i = 0; i < m->nff; i++)
        for (int j = 0; j < m->nff; j++) d.emplace_back(m->ffR[2 * i] - m->ffR[2 * j], m->ffR[2 * i + 1] - m->ffR[2 * j + 1]);
    std::sort(d.begin(), d.end());
    d.erase(std::unique(d.begin(), d.end()), d.end());
    m->nd = (int)d.size();
    m->deltas.clear();
    for (auto &p : d) { m->deltas.push_back(p.first); m->deltas.push_back(p.second); }
    std::vector<int> xs, ys;
    for (auto &p : d) { xs.push_back(p.first); ys.push_back(p.second); }
    std::sort(xs.begin(), xs.end()); xs.erase(std::unique(xs.begin(), xs.end()), xs.end());
    std::sort(ys.begin(), ys.end()); ys.erase(std::unique(ys.begin(), ys.end()), ys.end());
    m->dxs = xs;
    m->dys = ys;
    std::vector<int> dyh;
    for (int v : ys) if (v >= 0) dyh.push_back(v);
    const int ndyh = (int)dyh.size();
    m->dslot.assign(m->nd, 0);
    for (int k = 0; k < m->nd; k++) {
        int dx = d[k].first, dy = d[k].second;
        if (!(dy > 0 || (dy == 0 && dx >= 0))) { dx = -dx; dy = -dy; }
        const int xi = (int)(std::find(xs.begin(), xs.end(), dx) - xs.begin());
        const int yi = (int)(std::find(dyh.begin(), dyh.end(), dy) - dyh.begin());
        m->dslot[k] = xi * ndyh + yi;
    }
    m->dpartner.assign(m->nd, -1);
    for (int k = 0; k < m->nd; k++) {
        std::pair<int, int> v(-d[k].first, -d[k].second);
        m->dpartner[k] = (int)(std::lower_bound(d.begin(), d.end(), v) - d.begin());
    }
    m->dij.assign(m->nff * m->nff, 0);
    for (int i = 0; i < m->nff; i++)
        for (int j = 0; j < m->nff; j++) {
            std::pair<int, int> v(m->ffR[2 * i] - m->ffR[2 * j], m->ffR[2 * i + 1] - m->ffR[2 * j + 1]);
            m->dij[i * m->nff + j] = (int)(std::lower_bound(d.begin(), d.end(), v) - d.begin());
        }
}

// Projection gather tables (Sec. 3.3): bond classes, phase vectors, per-(R,R') term lists.
void build_gather_tables(tufrg_model *m)
{
    const int L = m->Lq, nff = m->nff;
    std::map<std::pair<int, int>, int> cls, phv;
    auto cls_of = [&](int x, int y) {
        std::pair<int, int> k(imod(x, L), imod(y, L));
        auto it = cls.find(k);
        if (it != cls.end()) return it->second;
        int id = (int)cls.size();
        cls[k] = id;
        return id;
    };
    auto ph_of = [&](int x, int y) {
        std::pair<int, int> k(imod(x, L), imod(y, L));
        auto it = phv.find(k);
        if (it != phv.end()) return it->second;
        int id = (int)phv.size();
        phv[k] = id;
        return id;
    };
    // classes of differences of two bonds, in a fixed enumeration order
    std::vector<std::pair<int, int>> clist;
    for (int i = 0; i < nff; i++)
        for (int j = 0; j < nff; j++) {
            const int x = imod(m->ffR[2 * i] - m->ffR[2 * j], L), y = imod(m->ffR[2 * i + 1] - m->ffR[2 * j + 1], L);
            if (cls.find({x, y}) == cls.end()) { cls_of(x, y); clist.emplace_back(x, y); }
        }
    for (int ch = 0; ch < 2; ch++) {
        m->gofs[ch].assign(nff * nff + 1, 0);
        m->gterms[ch].clear();
        m->gtab_export[ch].clear();
    }
    auto add = [&](int ch, int iR, int iRp, int kind, int cx, int cy, int i1, int i2, int px, int py) {
        GatherTerm t;
        t.cls = cls_of(cx, cy);
        t.i1 = i1;
        t.i2 = i2;
        t.ph = ph_of(px, py);
        t.kind = kind;
        m->gterms[ch].push_back(t);
        const int ex[9] = {iR, iRp, kind, imod(cx, L), imod(cy, L), i1, i2, imod(px, L), imod(py, L)};
        m->gtab_export[ch].insert(m->gtab_export[ch].end(), ex, ex + 9);
    };
    for (int iR = 0; iR < nff; iR++)
        for (int iRp = 0; iRp < nff; iRp++) {
            const int Rx = m->ffR[2 * iR], Ry = m->ffR[2 * iR + 1], Px = m->ffR[2 * iRp], Py = m->ffR[2 * iRp + 1];
            // P output
            for (auto &c : clist) {
                const int i1 = ff_index_mod(m, Rx + c.first, Ry + c.second);
                if (i1 < 0) continue;
                const int i2 = ff_index_mod(m, Px - c.first, Py - c.second);
                if (i2 >= 0) add(0, iR, iRp, 0, c.first, c.second, i1, i2, c.first, c.second);
                const int j2 = ff_index_mod(m, -Px - c.first, -Py - c.second);
                if (j2 >= 0) add(0, iR, iRp, 1, c.first, c.second, i1, j2, Px + c.first, Py + c.second);
            }
            m->gofs[0][iR * nff + iRp + 1] = (int)m->gterms[0].size();
            // C output
            for (auto &c : clist) {
                const int i1 = ff_index_mod(m, Rx + c.first, Ry + c.second);
                const int i2 = ff_index_mod(m, Px - c.first, Py - c.second);
                if (i1 >= 0 && i2 >= 0) add(1, iR, iRp, 2, c.first, c.second, i1, i2, c.first, c.second);
            }
            for (int i2 = 0; i2 < nff; i2++) {
                const int Wx = m->ffR[2 * i2], Wy = m->ffR[2 * i2 + 1];
                const int i1 = ff_index_mod(m, Rx - Px + Wx, Ry - Py + Wy);
                if (i1 >= 0) add(1, iR, iRp, 3, -Px, -Py, i1, i2, Wx, Wy);
            }
            m->gofs[1][iR * nff + iRp + 1] = (int)m->gterms[1].size();
        }
    m->ncls = (int)cls.size();
    m->cls.assign(2 * m->ncls, 0);
    for (auto &kv : cls) { m->cls[2 * kv.second] = kv.first.first; m->cls[2 * kv.second + 1] = kv.first.second; }
    m->nph = (int)phv.size();
    m->phv.assign(2 * m->nph, 0);
    for (auto &kv : phv) { m->phv[2 * kv.second] = kv.first.first; m->phv[2 * kv.second + 1] = kv.first.second; }
}

// The projection gather terms flattened per output matrix entry (same terms, same order as the
// per-(R, R') lists): for output channel ch and entry (row, col) = ((R, a), (R', b)), each term is
// the flat index of its source entry in the Fourier transforms [2][ncls][M][M] (high bit set when
// the term enters with a minus sign) and its phase-table column.  The orbital index pairs follow the
// channel layouts: P rows (s1,s2), columns (s4,s3); C rows (s1,s3), columns (s4,s2).
void build_entry_tables(const tufrg_model *m, std::vector<int> ofs[2], std::vector<int2> terms[2],
                        std::vector<double2> v0d[2])
{
    const int ns = m->ns, ns2 = ns * ns, nff = m->nff, M = m->M;
    const long M2 = (long)M * M;
    for (int ch = 0; ch < 2; ch++) {
        ofs[ch].assign(M2 + 1, 0);
        terms[ch].clear();
        v0d[ch].assign(M2, make_double2(0.0, 0.0));
        for (int row = 0; row < M; row++)
            for (int col = 0; col < M; col++) {
                const int iR = row / ns2, rp = row % ns2, iRp = col / ns2, cp = col % ns2;
                int s1, s2, s3, s4;
                if (ch == 0) { s1 = rp / ns; s2 = rp % ns; s4 = cp / ns; s3 = cp % ns; }
                else         { s1 = rp / ns; s3 = rp % ns; s4 = cp / ns; s2 = cp % ns; }
                if (iR == 0 && iRp == 0) {
                    const int v = ((s1 * ns + s2) * ns + s3) * ns + s4;
                    v0d[ch][(long)row * M + col] = make_double2(m->V0[2 * v], m->V0[2 * v + 1]);
                }
                const int pair = iR * nff + iRp;
                for (int t = m->gofs[ch][pair]; t < m->gofs[ch][pair + 1]; t++) {
                    const tufrg::GatherTerm &g = m->gterms[ch][t];
                    int sch, sr, sc;
                    bool neg;
                    switch (g.kind) {
                    case 0: sch = 1; sr = s1 * ns + s3; sc = s4 * ns + s2; neg = false; break;   // P <- C
                    case 1: sch = 1; sr = s1 * ns + s4; sc = s3 * ns + s2; neg = true; break;    // P <- D
                    case 2: sch = 0; sr = s1 * ns + s2; sc = s4 * ns + s3; neg = false; break;   // C <- P
                    default: sch = 1; sr = s1 * ns + s4; sc = s3 * ns + s2; neg = true; break;   // C <- D
                    }
                    const long idx = ((long)sch * m->ncls + g.cls) * M2 + (long)(g.i1 * ns2 + sr) * M + g.i2 * ns2 + sc;
                    terms[ch].push_back(make_int2((int)idx | (neg ? INT_MIN : 0), g.ph));
                }
                ofs[ch][(long)row * M + col + 1] = (int)terms[ch].size();
            }
    }
}

// ---- loop symmetries
// A unitary symmetry (G, U) of the hoppings, t_{G R} = U t_R U^dagger, maps the band projectors as
// P_l(G k) = U P_l(k) U^dagger and the loops as Lc(G q)[G Delta] = V Lc(q)[Delta] V^dagger with
// V = U (x) U on the P pair index (t2, t1) and V = U (x) U^* on the C pair index (t1, t2).  Time
// reversal, t_R = W t_R^* W^T, gives Lc(-q)[Delta] = V conj(Lc(q)[Delta]) V^dagger with V = W (x) W (P)
// and W (x) W^* (C); composed with (G, U) it maps q -> -G q, Delta -> G Delta.
// States are orbital (x) spin-1/2, index 2 * orbital + spin.  Candidates: the eight point operations of
// the square lattice, each with U = (signed permutation of the orbitals) (x) (diag(1, i^n) or
// antidiag(1, i^n) on the spin), and W = 1 (x) i sigma_y.  Every U, W and hence every V is monomial
// (one entry of modulus one per row), which is how they are stored: row i has its entry in column
// perm[i] with value ph[i] (global phases drop out of V . V^dagger).
struct LoopSymmetry {
    std::vector<int> list, dinv;
    std::vector<int2> qmap;
    std::vector<tufrg::SymElem> elem;
    std::vector<int> ffinv;   // [elem][nff] source bond of each target bond (G R_src = R_target), -1 if none
};

struct Mono {
    std::vector<int> perm;
    std::vector<std::complex<double>> ph;
};

void build_loop_symmetry(const tufrg_model *m, LoopSymmetry &ls)
{
    using cd = std::complex<double>;
    const int Gs[8][4] = {{1, 0, 0, 1}, {0, -1, 1, 0}, {-1, 0, 0, -1}, {0, 1, -1, 0},
                          {-1, 0, 0, 1}, {1, 0, 0, -1}, {0, 1, 1, 0}, {0, -1, -1, 0}};
    const int L = m->Lq, nd = m->nd, ns = m->ns, ns2 = ns * ns, norb = ns / 2;
    if (ns % 2 != 0 || ns2 > tufrg::SYM_MAXNS2) return;
    auto hop = [&](int h, int i, int j) {
        const size_t o = 2 * ((size_t)h * ns2 + (size_t)i * ns + j);
        return cd(m->hopt[o], m->hopt[o + 1]);
    };
    auto find_hop = [&](int x, int y) {
        for (int h = 0; h < m->nhop; h++)
            if (m->hopR[2 * h] == x && m->hopR[2 * h + 1] == y) return h;
        return -1;
    };
    auto find_delta = [&](int x, int y) {
        for (int k = 0; k < nd; k++)
            if (m->deltas[2 * k] == x && m->deltas[2 * k + 1] == y) return k;
        return -1;
    };
    double tmax = 0.0;
    for (int h = 0; h < m->nhop; h++)
        for (int i = 0; i < ns; i++)
            for (int j = 0; j < ns; j++) tmax = std::max(tmax, std::abs(hop(h, i, j)));
    const double tol = 1e-12 * std::max(1.0, tmax);
    // (U t U^dagger)_{ij} = ph_i t_{perm i, perm j} conj(ph_j) for a monomial U
    auto conj_ok = [&](const Mono &U, int h_from, int h_to, bool antiunitary) {
        for (int i = 0; i < ns; i++)
            for (int j = 0; j < ns; j++) {
                cd t = hop(h_from, U.perm[i], U.perm[j]);
                if (antiunitary) t = std::conj(t);
                if (std::abs(U.ph[i] * t * std::conj(U.ph[j]) - hop(h_to, i, j)) > tol) return false;
            }
        return true;
    };
    // orbital signed permutations (x) spin monomials
    std::vector<Mono> cands;
    {
        std::vector<int> p(norb);
        for (int i = 0; i < norb; i++) p[i] = i;
        do {
            for (int sg = 0; sg < (1 << norb); sg++)
                for (int c = 0; c < 8; c++) {
                    const cd sp = std::pow(cd(0.0, 1.0), c / 2);
                    Mono U;
                    U.perm.resize(ns);
                    U.ph.resize(ns);
                    for (int o = 0; o < norb; o++)
                        for (int s = 0; s < 2; s++) {
                            const int row = 2 * o + s;
                            const int scol = c % 2 == 0 ? s : 1 - s;   // diag(1, i^n) or antidiag(1, i^n)
                            const cd sph = s == 0 ? cd(1.0) : sp;
                            U.perm[row] = 2 * p[o] + scol;
                            U.ph[row] = ((sg >> o) & 1 ? -1.0 : 1.0) * sph;
                        }
                    cands.push_back(U);
                }
        } while (std::next_permutation(p.begin(), p.end()));
    }
    struct Op { int Gq[4], Gd[4]; Mono U; int conj; };
    std::vector<Op> ops;
    for (const int *G : Gs) {
        bool deltas_ok = true;
        for (int k = 0; k < nd && deltas_ok; k++)
            deltas_ok = find_delta(G[0] * m->deltas[2 * k] + G[1] * m->deltas[2 * k + 1],
                                   G[2] * m->deltas[2 * k] + G[3] * m->deltas[2 * k + 1]) >= 0;
        if (!deltas_ok) continue;
        std::vector<int> img(m->nhop, -1);
        bool hops_ok = true;
        for (int h = 0; h < m->nhop && hops_ok; h++) {
            img[h] = find_hop(G[0] * m->hopR[2 * h] + G[1] * m->hopR[2 * h + 1], G[2] * m->hopR[2 * h] + G[3] * m->hopR[2 * h + 1]);
            hops_ok = img[h] >= 0;
        }
        if (!hops_ok) continue;
        for (const Mono &U : cands) {
            bool ok = true;
            for (int h = 0; h < m->nhop && ok; h++) ok = conj_ok(U, h, img[h], false);   // t_{GR} = U t_R U^dagger
            if (!ok) continue;
            Op o{};
            std::copy(G, G + 4, o.Gq);
            std::copy(G, G + 4, o.Gd);
            o.U = U;
            o.conj = 0;
            ops.push_back(o);
            break;
        }
    }
    // time reversal W = 1 (x) i sigma_y: rows (2o, 2o+1) -> columns (2o+1, 2o) with values (1, -1)
    Mono W;
    W.perm.resize(ns);
    W.ph.resize(ns);
    for (int o = 0; o < norb; o++) {
        W.perm[2 * o] = 2 * o + 1; W.ph[2 * o] = 1.0;
        W.perm[2 * o + 1] = 2 * o; W.ph[2 * o + 1] = -1.0;
    }
    bool trs = true;
    for (int h = 0; h < m->nhop && trs; h++) trs = conj_ok(W, h, h, true);   // t_R = W t_R^* W^T
    // pair-index representation of V for a monomial U (P: a = t2 ns + t1 with U (x) U; C: a = t1 ns + t2 with U (x) U^*)
    auto pairV = [&](const Mono &U, int ch) {
        Mono V;
        V.perm.resize(ns2);
        V.ph.resize(ns2);
        for (int a = 0; a < ns2; a++) {
            const int x = a / ns, y = a % ns;
            V.perm[a] = U.perm[x] * ns + U.perm[y];
            V.ph[a] = ch == 0 ? U.ph[x] * U.ph[y] : U.ph[x] * std::conj(U.ph[y]);
        }
        return V;
    };
    struct Elem { int Gq[4], Gd[4]; Mono V[2]; int conj; };
    std::vector<Elem> elems;
    for (const Op &o : ops) {
        Elem e{};
        std::copy(o.Gq, o.Gq + 4, e.Gq);
        std::copy(o.Gd, o.Gd + 4, e.Gd);
        e.V[0] = pairV(o.U, 0);
        e.V[1] = pairV(o.U, 1);
        e.conj = 0;
        elems.push_back(e);
    }
    if (trs) {
        const Mono VT[2] = {pairV(W, 0), pairV(W, 1)};
        const size_t nu = elems.size();
        for (size_t i = 0; i < nu; i++) {
            Elem e{};
            for (int k = 0; k < 4; k++) { e.Gq[k] = -elems[i].Gq[k]; e.Gd[k] = elems[i].Gd[k]; }
            for (int ch = 0; ch < 2; ch++) {   // V_T conj(V_g): row a -> perm_g(perm_T(a)), ph_T(a) conj(ph_g(perm_T(a)))
                e.V[ch].perm.resize(ns2);
                e.V[ch].ph.resize(ns2);
                for (int a = 0; a < ns2; a++) {
                    const int b = VT[ch].perm[a];
                    e.V[ch].perm[a] = elems[i].V[ch].perm[b];
                    e.V[ch].ph[a] = VT[ch].ph[a] * std::conj(elems[i].V[ch].ph[b]);
                }
            }
            e.conj = 1;
            elems.push_back(e);
        }
    }
    // device tables: target a' reads source perm[a'] with phase i^qt[a']
    for (const Elem &el : elems) {
        tufrg::SymElem e{};
        e.conj = el.conj;
        for (int ch = 0; ch < 2; ch++)
            for (int a2 = 0; a2 < ns2; a2++) {
                const cd v = el.V[ch].ph[a2];
                e.src[ch][a2] = el.V[ch].perm[a2];
                e.qt[ch][a2] = std::abs(v - 1.0) < 1e-9 ? 0 : std::abs(v - cd(0, 1)) < 1e-9 ? 1
                             : std::abs(v + 1.0) < 1e-9 ? 2 : 3;
            }
        ls.elem.push_back(e);
        std::vector<int> inv(nd, 0);   // Delta_d' = G Delta_d  ->  inv[d'] = d
        for (int k = 0; k < nd; k++)
            inv[find_delta(el.Gd[0] * m->deltas[2 * k] + el.Gd[1] * m->deltas[2 * k + 1],
                           el.Gd[2] * m->deltas[2 * k] + el.Gd[3] * m->deltas[2 * k + 1])] = k;
        ls.dinv.insert(ls.dinv.end(), inv.begin(), inv.end());
        std::vector<int> finv(m->nff, -1);   // bonds: R_target = G R_source (modulo Lq)
        for (int i = 0; i < m->nff; i++) {
            const int x = el.Gd[0] * m->ffR[2 * i] + el.Gd[1] * m->ffR[2 * i + 1];
            const int y = el.Gd[2] * m->ffR[2 * i] + el.Gd[3] * m->ffR[2 * i + 1];
            const int j = ff_index_mod(m, x, y);
            if (j >= 0) finv[j] = i;
        }
        ls.ffinv.insert(ls.ffinv.end(), finv.begin(), finv.end());
    }
    // orbits: the smallest momentum of each orbit is its representative
    ls.qmap.assign(m->Nq, make_int2(-1, -1));
    for (int q = 0; q < m->Nq; q++) {
        if (ls.qmap[q].x >= 0) continue;
        const int pos = (int)ls.list.size();
        ls.list.push_back(q);
        const int qx = q / L, qy = q % L;
        for (size_t e = 0; e < elems.size(); e++) {
            const int *G = elems[e].Gq;
            const int x = ((G[0] * qx + G[1] * qy) % L + L) % L, y = ((G[2] * qx + G[3] * qy) % L + L) % L;
            const int q2 = x * L + y;
            if (ls.qmap[q2].x < 0) ls.qmap[q2] = make_int2(pos, (int)e);
        }
    }
}

// Autotuner decisions, shared by every model of the same shape in the process: the first model of a
// shape times the alternatives, later ones reuse its choice, so that equal models take equal paths (and
// give equal results) whatever the timing noise.  Key: device, decision kind and the sizes the costs
// depend on.
struct TuneResult {
    double ms[2];
    int choice;
    std::vector<double> cand_ms;   // launch-shape candidates: one time per candidate
    int aux = 0;                   // products: the chosen column-tile count
};
std::mutex g_tune_mutex;
std::map<std::vector<int>, TuneResult> g_tune_cache;

std::vector<int> tune_key(const tufrg_model *m, int kind)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return {dev, kind, m->precision, m->ns, m->M, m->Lq, m->nc, m->nd, m->nff, m->n_loop_q, m->n_sym_elem,
            m->d_sym_emap ? 1 : 0};
}

bool tune_lookup(const tufrg_model *m, int kind, TuneResult *r)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(tune_key(m, kind));
    if (it == g_tune_cache.end()) return false;
    *r = it->second;
    return true;
}

void tune_store(const tufrg_model *m, int kind, const TuneResult &r)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache.emplace(tune_key(m, kind), r);   // a concurrent first store wins
}

// e^{i q.R} for every coarse q and every listed vector (exact lattice phases).
std::vector<double2> phase_table(int Lq, const std::vector<int> &vecs)
{
    const int n = (int)vecs.size() / 2, Nq = Lq * Lq;
    std::vector<double2> t((size_t)Nq * n);
    for (int q = 0; q < Nq; q++)
        for (int c = 0; c < n; c++) {
            const long k = ((long)(q / Lq) * vecs[2 * c] + (long)(q % Lq) * vecs[2 * c + 1]) % Lq;
            const double a = 2.0 * M_PI * (double)((k + Lq) % Lq) / (double)Lq;
            t[(size_t)q * n + c] = make_double2(std::cos(a), std::sin(a));
        }
    return t;
}

}  // namespace
namespace tufrg {
// the captured right-hand-side graphs are dropped whenever the launches they hold would change
void drop_rhs_graphs(tufrg_model *m)
{
    for (auto &r : m->rhs_graphs)
        if (r.exec) cudaGraphExecDestroy(r.exec);
    m->rhs_graphs.clear();
}
}  // namespace tufrg
namespace {

void release(tufrg_model *m)
{
    void *ptrs[] = {m->d_E, m->d_U, m->d_U32, m->d_ft, m->d_ft32, m->d_dslot, m->d_deltas, m->d_hopR, m->d_hopt,
                    m->d_dij, m->d_gofs[0], m->d_gofs[1], m->d_gterms[0], m->d_gterms[1], m->d_ph, m->d_clsph,
                    m->d_V0, m->d_Lc, m->d_Lc32, m->d_part, m->d_Xr, m->d_A, m->d_A32, m->d_T, m->d_amax,
                    m->d_red, m->d_y, m->d_yt, m->d_yn, m->d_state_in, m->d_state_out, m->d_rec, m->d_Xr32,
                    m->d_ph32, m->d_dftpart, m->d_dpartner, m->d_err, m->d_scal, m->d_flow, m->d_eofs[0],
                    m->d_eofs[1], m->d_eterms[0], m->d_eterms[1], m->d_v0d[0], m->d_v0d[1], m->d_X32,
                    m->d_loop_list, m->d_qmap, m->d_sym_elem, m->d_sym_dinv, m->d_lph32,
                    m->d_clsph32, m->d_v0d32[0], m->d_v0d32[1], m->d_sym_srow, m->d_sym_qrow, m->d_sym_sinv, m->d_orb_ofs, m->d_orb_q, m->d_sym_emap, m->d_orb_lexp, m->d_band_tc,
                    m->d_dft_tabs, m->d_dft_phy, m->d_dft_phx, m->d_dft_phy32, m->d_dft_phx32, m->d_loop_w,
                    m->d_shard_q, m->d_shard_out, m->d_v0q, m->d_v0q32, m->d_ffW, m->d_amax_ch};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &p : m->d_k)
        if (p) cudaFree(p);
    for (auto &e : m->evpool) cudaEventDestroy(e);
    m->evpool.clear();
    tufrg_set_surrogate(m, nullptr, nullptr, nullptr, nullptr, 0.0, 0, nullptr);
    if (m->h_flow) cudaFreeHost(m->h_flow);
    if (m->step_graph) cudaGraphExecDestroy(m->step_graph);
    drop_rhs_graphs(m);
    for (auto &e : m->rhs_ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : m->aux_ev)
        if (e) cudaEventDestroy(e);
    if (m->aux_stream) cudaStreamDestroy(m->aux_stream);
    if (m->rhs_stream) cudaStreamDestroy(m->rhs_stream);
    if (m->flow_ev) cudaEventDestroy(m->flow_ev);
    if (m->flow_stream) cudaStreamDestroy(m->flow_stream);
    for (int b = 0; b < 2; b++) {
        if (m->d_bin[b]) cudaFree(m->d_bin[b]);
        if (m->d_bout[b]) cudaFree(m->d_bout[b]);
        if (m->ev_in[b]) cudaEventDestroy(m->ev_in[b]);
        if (m->ev_comp[b]) cudaEventDestroy(m->ev_comp[b]);
        if (m->ev_out[b]) cudaEventDestroy(m->ev_out[b]);
    }
    if (m->s_h2d) cudaStreamDestroy(m->s_h2d);
    if (m->s_d2h) cudaStreamDestroy(m->s_d2h);
}

size_t state_elems(const tufrg_model *m) { return (size_t)2 * m->Nq * m->M * m->M; }

// One evaluation of the right-hand side into d_out at the temperature held in m->d_scal[0],
// each channel scaled by c_X * m->d_scal[1] (1 for dX/dT, T for the flow variable ln T).
// The split path evaluates on an FP32 copy of the state: d_state32 when the caller has already
// written one (the flow's stage combinations do), else a conversion of d_state into m->d_X32.
tufrg_status rhs_device(tufrg_model *m, const double2 *d_state, int mask, double2 *d_out, const float2 *d_state32,
                        bool symmetric_state)
{
    const bool split = m->precision != TUFRG_FP64;
    // a symmetric state needs projections and products at the orbit representatives only
    const bool sym = symmetric_state && m->sym_state;
    const int *ql = sym ? m->d_loop_list : nullptr;
    const int nl = sym ? m->n_loop_q : 0;
    // The state's branch (Fourier transform, projections) and the loops' branch (Fermi data, loop k-sum and its
    // reduction) share no buffer: on a second stream they overlap, joined before the products.  Serial while the
    // phases are timed (their events stay on one stream).
    const bool fork = !m->timing && m->aux_stream;
    auto state_branch = [&]() -> tufrg_status {
        // without an FP32 copy the separable transform writes one as it reads the FP64 state (the sliced
        // direct transform reads a converted copy)
        if (split && !d_state32 && m->dft_warps == 0) {
            CK(launch_to_f32(m, d_state, m->d_X32, state_elems(m)), "state conversion");
            d_state32 = m->d_X32;
        }
        CK(launch_dft(m, d_state, d_state32, mask), "Fourier transform");
        if (split && !d_state32) d_state32 = m->d_X32;
        // the split path's products read the FP32 copy only
        CK(launch_project(m, d_state, d_state32, mask, split ? nullptr : m->d_A, ql, nl), "projections");
        return TUFRG_OK;
    };
    if (fork) {
        CK(cudaEventRecord(m->aux_ev[0], m->stream), "fork");
        CK(cudaStreamWaitEvent(m->aux_stream, m->aux_ev[0], 0), "fork");
        const cudaStream_t main = m->stream;
        m->stream = m->aux_stream;
        const tufrg_status st = state_branch();
        m->stream = main;
        if (st != TUFRG_OK) return st;
        CK(cudaEventRecord(m->aux_ev[1], m->aux_stream), "join");
    }
    CK(launch_fermi(m), "fermi tables");
    // a symmetric state's products read the loops of the orbit representatives only
    CK(launch_loops(m, mask, sym), "loop k-sum");
    if (fork) {
        CK(cudaStreamWaitEvent(m->stream, m->aux_ev[1], 0), "join");
    } else {
        const tufrg_status st = state_branch();
        if (st != TUFRG_OK) return st;
    }
    if (sym) CK(launch_products_sym(m, mask, d_out), "V.L.V products (orbit representatives)");
    else CK(launch_vlv(m, m->d_A, mask, d_out), "V.L.V products");
    return TUFRG_OK;
}

// Dormand-Prince 5(4) tableau (stage nodes c, coefficients a, error weights b - b*)
const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
const double DP_A[7][6] = {
    {0},
    {1.0 / 5},
    {3.0 / 40, 9.0 / 40},
    {44.0 / 45, -56.0 / 15, 32.0 / 9},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
    {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
const double DP_E[7] = {35.0 / 384 - 5179.0 / 57600, 0.0, 500.0 / 1113 - 7571.0 / 16695, 125.0 / 192 - 393.0 / 640,
                        -2187.0 / 6784 + 92097.0 / 339200, 11.0 / 84 - 187.0 / 2100, -1.0 / 40};

// Enqueue one Dormand-Prince attempt on the model's stream: six stage right-hand sides, the error
// norm, the accept/reject decision and the FSAL commit, all driven by the device flow state.
tufrg_status enqueue_attempt(tufrg_model *m, int mask)
{
    const size_t n = state_elems(m);
    double2 *k[7];
    for (int i = 0; i < 7; i++) k[i] = m->d_k[i];
    const bool split = m->precision != TUFRG_FP64;
    for (int j = 1; j < 7; j++) {
        // the stage states are FP64 (and only the last one, the candidate solution, is kept); on the
        // split path the combination writes the FP32 copy that the evaluation reads instead
        double2 *dst = j == 6 ? m->d_yn : (split ? nullptr : m->d_yt);
        CK(launch_rk_combine(m, dst, split ? m->d_X32 : nullptr, m->d_y, m->d_flow, DP_A[j], k, j, n), "stage combination");
        CK(launch_stage_scalars(m, m->d_flow, DP_C[j]), "stage temperature");
        tufrg_status st = rhs_device(m, dst, mask, k[j], split ? m->d_X32 : nullptr, true);
        if (st != TUFRG_OK) return st;
    }
    CK(launch_rk_error(m, m->d_y, m->d_yn, m->d_flow, DP_E, k, 7, n), "error norm");
    CK(launch_flow_decide(m, m->d_flow), "step decision");
    CK(launch_flow_commit(m, m->d_flow, m->d_y, m->d_yn, k[0], k[6], n), "step commit");
    return TUFRG_OK;
}

// The flow's buffers: state, candidate, stage derivatives, device controller and its pinned host mirror.
tufrg_status flow_alloc(tufrg_model *m)
{
    const size_t n = state_elems(m);
    if (!m->d_y) {
        CK(dalloc(&m->d_y, n), "cudaMalloc flow state");
        CK(dalloc(&m->d_yt, n), "cudaMalloc flow state");
        CK(dalloc(&m->d_yn, n), "cudaMalloc flow state");
        for (auto &k : m->d_k) CK(dalloc(&k, n), "cudaMalloc flow stages");
        CK(dalloc(&m->d_flow, 1), "cudaMalloc flow state");
        CK(cudaMallocHost(reinterpret_cast<void **>(&m->h_flow), sizeof(FlowDev)), "cudaMallocHost flow state");
    }
    return TUFRG_OK;
}

// Capture one Dormand-Prince attempt of the given channel mask as the model's step graph (kept while the mask and
// the launch shapes stay the same).
tufrg_status flow_capture(tufrg_model *m, int mask)
{
    if (m->step_graph && m->step_graph_mask == mask) return TUFRG_OK;
    if (m->step_graph) {
        cudaGraphExecDestroy(m->step_graph);
        m->step_graph = nullptr;
    }
    const bool timing = m->timing;
    m->timing = false;   // no event records inside the captured graph
    const long long l0 = m->launches, ll0 = m->loop_launches;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    tufrg_status st = enqueue_attempt(m, mask);
    cudaError_t ce = cudaStreamEndCapture(m->stream, &g);
    m->timing = timing;
    m->launches = l0;
    m->loop_launches = ll0;
    if (st != TUFRG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return cuda_fail(m, ce, "end capture");
    ce = cudaGraphInstantiate(&m->step_graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(m, ce, "graph instantiate");
    m->step_graph_mask = mask;
    return TUFRG_OK;
}

// Allocate the flow buffers, zero the state, evaluate k1 = f(y0) and capture one attempt as a graph.
tufrg_status flow_prepare(tufrg_model *m, const tufrg_flow_opts *o)
{
    const size_t n = state_elems(m);
    tufrg_status st = flow_alloc(m);
    if (st != TUFRG_OK) return st;
    FlowDev f{};
    f.x = std::log(o->T0);
    f.xend = std::log(o->T_end);
    f.h = o->h0;
    if (f.x + f.h < f.xend) f.h = f.xend - f.x;
    f.x_prev = f.x;
    f.atol = o->atol;
    f.rtol = o->rtol;
    f.stop = o->stop;
    f.max_tries = o->max_steps;
    f.Tc = o->T_end;
    *m->h_flow = f;
    CK(cudaMemcpyAsync(m->d_flow, m->h_flow, sizeof(FlowDev), cudaMemcpyHostToDevice, m->stream), "copy flow state");
    CK(cudaMemsetAsync(m->d_y, 0, sizeof(double2) * n, m->stream), "zero state");
    CK(surrogate_rearm(m), "re-arm surrogate");
    // k1 = f(x0, y0) and max|A| of the initial state
    CK(launch_stage_scalars(m, m->d_flow, 0.0), "stage temperature");
    st = rhs_device(m, m->d_y, o->channel_mask, m->d_k[0], nullptr, true);
    if (st != TUFRG_OK) return st;
    CK(launch_flow_init(m, m->d_flow), "flow init");
    if ((st = flow_capture(m, o->channel_mask)) != TUFRG_OK) return st;
    // the controller state after the initial evaluation: a flow whose initial max|A| already exceeds the stop
    // value is critical at T0 and runs no attempt
    CK(cudaMemcpyAsync(m->h_flow, m->d_flow, sizeof(FlowDev), cudaMemcpyDeviceToHost, m->stream), "copy flow state");
    CK(cudaStreamSynchronize(m->stream), "sync");
    return TUFRG_OK;
}

// Flows run on a private non-blocking stream (the legacy default stream cannot be captured);
// it is ordered after the user's stream on entry and the user's stream after it on exit.
tufrg_status flow_enter(tufrg_model *m, cudaStream_t *user)
{
    *user = m->stream;
    if (!m->flow_stream) {
        CK(cudaStreamCreateWithFlags(&m->flow_stream, cudaStreamNonBlocking), "create flow stream");
        CK(cudaEventCreateWithFlags(&m->flow_ev, cudaEventDisableTiming), "create flow event");
    }
    CK(cudaEventRecord(m->flow_ev, m->stream), "record");
    CK(cudaStreamWaitEvent(m->flow_stream, m->flow_ev, 0), "wait");
    m->stream = m->flow_stream;
    return TUFRG_OK;
}

tufrg_status flow_leave(tufrg_model *m, cudaStream_t user)
{
    m->stream = user;
    CK(cudaEventRecord(m->flow_ev, m->flow_stream), "record");
    CK(cudaStreamWaitEvent(user, m->flow_ev, 0), "wait");
    return TUFRG_OK;
}

tufrg_status flow_check_args(tufrg_model *m, const tufrg_flow_opts *o, tufrg_flow_result *res)
{
    if (!m || !o || !res) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!(o->T0 > o->T_end) || !(o->T_end > 0)) return fail(m, TUFRG_EINVAL, "need T0 > T_end > 0");
    if (!(o->rtol > 0) || !(o->atol >= 0) || !(o->h0 < 0)) return fail(m, TUFRG_EINVAL, "bad tolerances or h0");
    if ((o->channel_mask & 3) == 0 || (o->channel_mask & ~3)) return fail(m, TUFRG_EINVAL, "bad channel_mask");
    if (o->max_steps < 1) return fail(m, TUFRG_EINVAL, "max_steps must be positive");
    return TUFRG_OK;
}

// Result of a finished flow: read the device state, locate the maximum of the last projection.
tufrg_status flow_finish(tufrg_model *m, void *d_state_out, tufrg_flow_result *res)
{
    const FlowDev &f = *m->h_flow;
    res->n_steps = f.n_steps;
    res->n_reject = f.n_reject;
    res->n_rhs = 1 + 6 * f.tries;
    res->amax = f.amax;
    res->T_last = std::exp(f.x);
    res->crossed = f.status == 1;
    res->Tc = res->crossed ? f.Tc : res->T_last;
    // the last stage-7 projection belongs to the last accepted state when the flow stopped on an accepted step
    const size_t nA = state_elems(m), M2 = (size_t)m->M * m->M;
    CK(launch_amax_locate(m, nA, m->sym_state), "locate maximum");
    unsigned long long b[4];
    CK(cudaMemcpyAsync(b, m->d_amax, sizeof(b), cudaMemcpyDeviceToHost, m->stream), "copy scalars");
    CK(cudaStreamSynchronize(m->stream), "sync");
    if (b[1] < nA) {
        res->lead_channel = (int)(b[1] / ((size_t)m->Nq * M2));
        res->lead_q = (int)((b[1] / M2) % m->Nq);
    }
    if (d_state_out)
        CK(cudaMemcpyAsync(d_state_out, m->d_y, sizeof(double2) * nA, cudaMemcpyDeviceToDevice, m->stream), "copy state out");
    CK(cudaStreamSynchronize(m->stream), "sync");
    switch (f.status) {
    case 3: return fail(m, TUFRG_ENOTCONV, "flow step limit reached");
    case 4: return fail(m, TUFRG_ENONFINITE, "non-finite right-hand side or error norm");
    case 5: return fail(m, TUFRG_ENOTCONV, "step size underflow");
    default: return TUFRG_OK;
    }
}

// Checkpoint layout: this header, the device controller (FlowDev), the state y and its derivative k1 = f(y) (the
// first stage of the next attempt), both [2][Nq][M][M] complex FP64.
struct CkptHeader {
    char magic[8];          // "TUFRGCK1"
    int version, flowdev_bytes;
    int precision, ns, nff, Lq, nc, M, channel_mask, basis, regulator, loops_tc;
    int products, ky_chunks;   // launch shapes in use (they fix the summation order)
    long long n_elems;
};

CkptHeader ckpt_header(const tufrg_model *m, int mask)
{
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "TUFRGCK1", 8);
    h.version = 1;
    h.flowdev_bytes = (int)sizeof(FlowDev);
    h.precision = m->precision;
    h.ns = m->ns;
    h.nff = m->nff;
    h.Lq = m->Lq;
    h.nc = m->nc;
    h.M = m->M;
    h.channel_mask = mask;
    h.basis = m->basis;
    h.regulator = m->regulator;
    h.loops_tc = m->loops_tc ? 1 : 0;
    h.products = m->products;
    h.ky_chunks = m->plan.ky_chunks;
    h.n_elems = (long long)state_elems(m);
    return h;
}

double bits_to_double(unsigned long long b)
{
    double d;
    std::memcpy(&d, &b, sizeof(d));
    return d;
}

tufrg_status read_device_error(tufrg_model *m)
{
    int dev_err = 0;
    CK(cudaMemcpy(&dev_err, m->d_err, sizeof(int), cudaMemcpyDeviceToHost), "copy error flag");
    if (dev_err) return fail(m, TUFRG_ETIMEOUT, "a bounded device-side wait gave up");
    return TUFRG_OK;
}

}  // namespace

extern "C" {

// The host tables of init grow with the meshes and the bond set (host_alloc_fail).
tufrg_status tufrg_init_model(const tufrg_model_desc *desc, void *cuda_stream, tufrg_model **out)
try {
    if (!out) return TUFRG_EINVAL;
    *out = nullptr;
    if (!desc) return TUFRG_EINVAL;
    tufrg_model *m = new (std::nothrow) tufrg_model();
    if (!m) return TUFRG_ENOMEM;
    *out = m;   // so that tufrg_last_error works even when set-up fails
    // an error that an earlier runtime call of this thread left pending (a failed allocation of the caller's) would
    // be taken for the failure of the first launch below; it is not this model's
    (void)cudaGetLastError();
    const tufrg_model_desc &d = *desc;
    if (d.n_s < 1 || d.n_s > 8) return fail(m, TUFRG_EINVAL, "n_s must be in [1, 8]");
    if (d.n_s != 2 && d.n_s != 4 && d.n_s != 6) return fail(m, TUFRG_ENOTSUP, "the library supports n_s = 2, 4, 6");
    if (d.n_hop < 1 || !d.hop_R || !d.hop_t) return fail(m, TUFRG_EINVAL, "empty hopping list");
    if (!d.V0) return fail(m, TUFRG_EINVAL, "V0 is NULL");
    if (d.n_ff < 1 || !d.ff_R) return fail(m, TUFRG_EINVAL, "empty bond set");
    if (d.ff_R[0] != 0 || d.ff_R[1] != 0) return fail(m, TUFRG_EINVAL, "ff_R[0] must be (0,0)");
    if (d.Lq < 2 || d.nc < 1) return fail(m, TUFRG_EINVAL, "Lq >= 2 and nc >= 1 required");
    if ((long)d.Lq * d.nc > 4096) return fail(m, TUFRG_EINVAL, "fine mesh too large");
    if (d.precision != TUFRG_FP64 && d.precision != TUFRG_SPLIT32) return fail(m, TUFRG_EINVAL, "unknown precision");
    if (d.products < TUFRG_PRODUCTS_AUTO || d.products > TUFRG_PRODUCTS_SIMT) return fail(m, TUFRG_EINVAL, "unknown products backend");
    if (d.loops < TUFRG_LOOPS_AUTO || d.loops > TUFRG_LOOPS_SIMT) return fail(m, TUFRG_EINVAL, "unknown loops backend");
    if (d.basis != TUFRG_BASIS_ORBITAL && d.basis != TUFRG_BASIS_BAND) return fail(m, TUFRG_EINVAL, "unknown basis");
    m->basis = d.basis;
    if (d.symmetry != TUFRG_SYMMETRY_AUTO && d.symmetry != TUFRG_SYMMETRY_OFF && d.symmetry != TUFRG_SYMMETRY_STATES)
        return fail(m, TUFRG_EINVAL, "unknown symmetry option");
    if (d.filling > 0 && !(d.T_mu > 0)) return fail(m, TUFRG_EINVAL, "T_mu must be > 0 when filling > 0");
    if (d.regulator != TUFRG_REG_TEMPERATURE && d.regulator != TUFRG_REG_MOMENTUM_SHELL)
        return fail(m, TUFRG_EINVAL, "unknown regulator");
    if (d.regulator == TUFRG_REG_MOMENTUM_SHELL && !(d.T_reg > 0 && std::isfinite(d.T_reg)))
        return fail(m, TUFRG_EINVAL, "the momentum-shell regulator needs T_reg > 0");
    m->regulator = d.regulator;
    m->T_reg = d.T_reg;
    m->ns = d.n_s; m->nhop = d.n_hop; m->nff = d.n_ff; m->Lq = d.Lq; m->nc = d.nc; m->precision = d.precision;
    m->Lf = d.Lq * d.nc; m->Nq = d.Lq * d.Lq; m->Nk = m->Lf * m->Lf; m->M = d.n_ff * d.n_s * d.n_s;
    m->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    m->hopR.assign(d.hop_R, d.hop_R + 2 * d.n_hop);
    m->hopt.assign(d.hop_t, d.hop_t + (size_t)2 * d.n_hop * d.n_s * d.n_s);
    m->V0.assign(d.V0, d.V0 + 2 * (size_t)d.n_s * d.n_s * d.n_s * d.n_s);
    m->ffR.assign(d.ff_R, d.ff_R + 2 * d.n_ff);
    // bonds must be distinct modulo Lq (otherwise the plane waves are not orthonormal on the mesh)
    for (int i = 0; i < m->nff; i++)
        for (int j = 0; j < i; j++)
            if (imod(m->ffR[2 * i] - m->ffR[2 * j], m->Lq) == 0 && imod(m->ffR[2 * i + 1] - m->ffR[2 * j + 1], m->Lq) == 0)
                return fail(m, TUFRG_EINVAL, "bonds are not distinct modulo Lq");
    // Hermiticity of H(k): t_{-R} = t_R^dagger
    const int ns = m->ns;
    for (int h = 0; h < m->nhop; h++) {
        int g = -1;
        for (int h2 = 0; h2 < m->nhop; h2++)
            if (m->hopR[2 * h2] == -m->hopR[2 * h] && m->hopR[2 * h2 + 1] == -m->hopR[2 * h + 1]) g = h2;
        if (g < 0) return fail(m, TUFRG_EINVAL, "hopping list lacks t_{-R} for some R");
        for (int i = 0; i < ns; i++)
            for (int j = 0; j < ns; j++) {
                const double *a = &m->hopt[2 * ((size_t)h * ns * ns + i * ns + j)];
                const double *b = &m->hopt[2 * ((size_t)g * ns * ns + j * ns + i)];
                if (std::fabs(a[0] - b[0]) > 1e-12 || std::fabs(a[1] + b[1]) > 1e-12)
                    return fail(m, TUFRG_EINVAL, "H(k) is not Hermitian: t_{-R} != t_R^dagger");
            }
    }
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev), "device attributes");

    build_loop_tables(m);
    build_gather_tables(m);
    build_irrep_basis(m);   // empty when the bond set is not closed under the point group
    // loop symmetries (TUFRG_SYMMETRY_AUTO, split two-band path)
    m->n_loop_q = m->Nq;
    if (m->basis == TUFRG_BASIS_BAND && !band_basis_supported(m))
        return fail(m, TUFRG_ENOTSUP, "the band-basis flow needs a two-band model with M <= 64");
    // the loop symmetries act on orbital indices; the band basis does not use them
    if (d.symmetry != TUFRG_SYMMETRY_OFF && m->basis == TUFRG_BASIS_ORBITAL &&
        ((ns == 2 && loops2_supported(m)) || (ns != 2 && loops_gen_supported(m)))) {
        LoopSymmetry ls;
        build_loop_symmetry(m, ls);
        if ((int)ls.list.size() < m->Nq) {
            m->sym = true;
            m->n_loop_q = (int)ls.list.size();
            m->n_sym_elem = (int)ls.elem.size();
            CK(upload(&m->d_loop_list, ls.list, m->stream), "upload symmetry tables");
            CK(upload(&m->d_qmap, ls.qmap, m->stream), "upload symmetry tables");
            CK(upload(&m->d_sym_elem, ls.elem, m->stream), "upload symmetry tables");
            CK(upload(&m->d_sym_dinv, ls.dinv, m->stream), "upload symmetry tables");
            // symmetric states: every element must map the bond set onto itself and leave the bare vertex's
            // onsite blocks invariant (a flow from X = 0 then stays symmetric)
            bool ok = true;
            for (int v : ls.ffinv) ok = ok && v >= 0;
            const int nsq = ns * ns;
            auto blk = [&](int ch, int a, int b) {   // onsite block of V0 in the channel's pair layout
                int s1, s2, s3, s4;
                if (ch == 0) { s1 = a / ns; s2 = a % ns; s4 = b / ns; s3 = b % ns; }
                else         { s1 = a / ns; s3 = a % ns; s4 = b / ns; s2 = b % ns; }
                const size_t o = 2 * ((((size_t)s1 * ns + s2) * ns + s3) * ns + s4);
                return std::complex<double>(m->V0[o], m->V0[o + 1]);
            };
            for (size_t e = 0; e < ls.elem.size() && ok; e++)
                for (int ch = 0; ch < 2 && ok; ch++)
                    for (int a2 = 0; a2 < nsq && ok; a2++)
                        for (int b2 = 0; b2 < nsq && ok; b2++) {
                            const tufrg::SymElem &el = ls.elem[e];
                            std::complex<double> v = blk(ch, el.src[ch][a2], el.src[ch][b2]);
                            if (el.conj) v = std::conj(v);
                            const int k = ((el.qt[ch][a2] - el.qt[ch][b2]) % 4 + 4) % 4;
                            v *= std::pow(std::complex<double>(0.0, 1.0), k);
                            ok = std::abs(v - blk(ch, a2, b2)) <= 1e-12 * (1.0 + std::abs(blk(ch, a2, b2)));
                        }
            if (ok) {
                // per element and channel: source row (= column) index and quarter turns of every target index
                std::vector<int> srow((size_t)ls.elem.size() * 2 * m->M), qrow((size_t)ls.elem.size() * 2 * m->M);
                for (size_t e = 0; e < ls.elem.size(); e++)
                    for (int ch = 0; ch < 2; ch++)
                        for (int r = 0; r < m->M; r++) {
                            const size_t o = (e * 2 + ch) * m->M + r;
                            srow[o] = ls.ffinv[e * m->nff + r / nsq] * nsq + ls.elem[e].src[ch][r % nsq];
                            qrow[o] = ls.elem[e].qt[ch][r % nsq];
                        }
                m->sym_state = true;
                CK(upload(&m->d_sym_srow, srow, m->stream), "upload symmetry tables");
                CK(upload(&m->d_sym_qrow, qrow, m->stream), "upload symmetry tables");
                // the inverse maps (every srow is a permutation when the bond set and the orbital pairs are closed
                // under the elements; otherwise the copy runs per target momentum)
                std::vector<int> sinv(srow.size(), -1);
                bool perm = true;
                for (size_t o = 0; o < srow.size() && perm; o++) {
                    const size_t base = o / m->M * m->M;
                    int &t = sinv[base + srow[o]];
                    perm = t < 0;
                    t = (int)(o - base);
                }
                if (perm) CK(upload(&m->d_sym_sinv, sinv, m->stream), "upload symmetry tables");
                std::vector<int> ofs(m->n_loop_q + 1, 0), oq(m->Nq);
                for (int q = 0; q < m->Nq; q++) ofs[ls.qmap[q].x + 1]++;
                int max_orbit = 0;
                for (int p = 0; p < m->n_loop_q; p++) max_orbit = std::max(max_orbit, ofs[p + 1]);
                for (int p = 0; p < m->n_loop_q; p++) ofs[p + 1] += ofs[p];
                // the momenta of every orbit, orbit after orbit (the copy of the representatives' products to the
                // other members runs in this order, so that a representative's matrix stays in L2 for its orbit)
                std::vector<int> fill(ofs.begin(), ofs.end() - 1);
                for (int q = 0; q < m->Nq; q++) oq[fill[ls.qmap[q].x]++] = q;
                CK(upload(&m->d_orb_ofs, ofs, m->stream), "upload symmetry tables");
                CK(upload(&m->d_orb_q, oq, m->stream), "upload symmetry tables");
                if (orbit_products_supported(m) && max_orbit <= orbit_max_size()) {
                    // fused orbit products: per element and channel, the source entry, quarter turns and
                    // conjugation of every target entry
                    const int M = m->M;
                    std::vector<int> emap((size_t)ls.elem.size() * 2 * M * M);
                    for (size_t e = 0; e < ls.elem.size(); e++)
                        for (int ch = 0; ch < 2; ch++) {
                            const int *sr = &srow[(e * 2 + ch) * M], *qr = &qrow[(e * 2 + ch) * M];
                            // i^k (conj ? conj(w) : w) as (swap, negate re, negate im), indexed [conj][k]
                            static const int compose[2][4] = {{0, 6, 3, 5}, {1, 4, 2, 7}};
                            for (int r = 0; r < M; r++)
                                for (int c = 0; c < M; c++)
                                    emap[((e * 2 + ch) * M + r) * M + c] =
                                        (sr[r] * M + sr[c]) << 3 | compose[ls.elem[e].conj ? 1 : 0][(qr[r] - qr[c]) & 3];
                        }
                    std::vector<int> lexp((size_t)M * M);
                    for (int r = 0; r < M; r++)
                        for (int c = 0; c < M; c++)
                            lexp[(size_t)r * M + c] = (m->dij[(r >> 2) * m->nff + (c >> 2)] * 4 + (r & 3)) * 4 + (c & 3);
                    CK(upload(&m->d_orb_lexp, lexp, m->stream), "upload symmetry tables");
                    CK(upload(&m->d_sym_emap, emap, m->stream), "upload symmetry tables");
                }
            }
        }
    }
    m->plan = plan_loops(m);
    // the two-band split loop kernel's launch shapes are timed at the end of the set-up (the partial sums are
    // sized for the largest)
    if (loops2_supported(m)) m->plan_cand = loop_plan_candidates(m);
    int max_partials = m->plan.n_partials;
    for (const LoopPlan &p : m->plan_cand) max_partials = std::max(max_partials, p.n_partials);

    // ---- device memory (and the right-hand side's second stream)
    CK(cudaStreamCreateWithFlags(&m->aux_stream, cudaStreamNonBlocking), "create stream");
    CK(cudaEventCreateWithFlags(&m->aux_ev[0], cudaEventDisableTiming), "create event");
    CK(cudaEventCreateWithFlags(&m->aux_ev[1], cudaEventDisableTiming), "create event");
    const size_t Nk = m->Nk, ns2 = (size_t)ns * ns, ns4 = ns2 * ns2, M2 = (size_t)m->M * m->M;
    const bool split = m->precision != TUFRG_FP64;
    std::vector<double2> hopt2((size_t)m->nhop * ns2), V02(ns4);
    for (size_t i = 0; i < hopt2.size(); i++) hopt2[i] = make_double2(m->hopt[2 * i], m->hopt[2 * i + 1]);
    for (size_t i = 0; i < V02.size(); i++) V02[i] = make_double2(m->V0[2 * i], m->V0[2 * i + 1]);
    CK(upload(&m->d_hopR, m->hopR, m->stream), "upload hoppings");
    CK(upload(&m->d_hopt, hopt2, m->stream), "upload hoppings");
    CK(upload(&m->d_V0, V02, m->stream), "upload V0");
    CK(upload(&m->d_deltas, m->deltas, m->stream), "upload bond tables");
    CK(upload(&m->d_dslot, m->dslot, m->stream), "upload bond tables");
    CK(upload(&m->d_dpartner, m->dpartner, m->stream), "upload bond tables");
    CK(upload(&m->d_dij, m->dij, m->stream), "upload bond tables");
    for (int ch = 0; ch < 2; ch++) {
        CK(upload(&m->d_gofs[ch], m->gofs[ch], m->stream), "upload gather tables");
        CK(upload(&m->d_gterms[ch], m->gterms[ch], m->stream), "upload gather tables");
    }
    if (2L * m->ncls * (long)m->M * m->M >= (long)INT_MAX) return fail(m, TUFRG_ETOOBIG, "projection tables exceed 2^31 entries");
    {
        std::vector<int> eofs[2];
        std::vector<int2> eterms[2];
        std::vector<double2> v0d[2];
        build_entry_tables(m, eofs, eterms, v0d);
        for (int ch = 0; ch < 2; ch++) {
            CK(upload(&m->d_eofs[ch], eofs[ch], m->stream), "upload projection tables");
            if (!eterms[ch].empty()) CK(upload(&m->d_eterms[ch], eterms[ch], m->stream), "upload projection tables");
            CK(upload(&m->d_v0d[ch], v0d[ch], m->stream), "upload projection tables");
            if (split) {
                std::vector<float2> v32(v0d[ch].size());
                for (size_t i = 0; i < v32.size(); i++) v32[i] = make_float2((float)v0d[ch][i].x, (float)v0d[ch][i].y);
                CK(upload(&m->d_v0d32[ch], v32, m->stream), "upload projection tables");
            }
        }
    }
    {
        std::vector<double2> ph = phase_table(m->Lq, m->phv);
        CK(upload(&m->d_ph, ph, m->stream), "upload phase table");
        if (split) {
            std::vector<float2> ph32(ph.size());
            for (size_t i = 0; i < ph.size(); i++) ph32[i] = make_float2((float)ph[i].x, (float)ph[i].y);
            CK(upload(&m->d_ph32, ph32, m->stream), "upload phase table");
        }
    }
    m->max_terms = 0;
    for (int ch = 0; ch < 2; ch++)
        for (int p = 0; p < m->nff * m->nff; p++)
            m->max_terms = std::max(m->max_terms, m->gofs[ch][p + 1] - m->gofs[ch][p]);
    m->dft_nsplit = dft_plan_nsplit(m);
    {
        // separable Fourier transform: the distinct R_y and R_x of the classes, classes grouped by R_y
        std::vector<int> ry, rx;
        for (int c = 0; c < m->ncls; c++) {
            if (std::find(ry.begin(), ry.end(), m->cls[2 * c + 1]) == ry.end()) ry.push_back(m->cls[2 * c + 1]);
            if (std::find(rx.begin(), rx.end(), m->cls[2 * c]) == rx.end()) rx.push_back(m->cls[2 * c]);
        }
        m->dft_nry = (int)ry.size();
        m->dft_nrx = (int)rx.size();
        dft_sep_plan(m, &m->dft_warps);
        if (m->dft_warps > 0) {
            std::vector<int> tabs(2 * m->ncls + m->dft_nry + 1, 0);
            int pos = 0;
            for (int r = 0; r < m->dft_nry; r++) {
                tabs[2 * m->ncls + r] = pos;
                for (int c = 0; c < m->ncls; c++)
                    if (m->cls[2 * c + 1] == ry[r]) {
                        tabs[pos] = c;
                        tabs[m->ncls + pos] = (int)(std::find(rx.begin(), rx.end(), m->cls[2 * c]) - rx.begin());
                        pos++;
                    }
            }
            tabs[2 * m->ncls + m->dft_nry] = pos;
            // e^{i 2 pi u R / Lq} with u R reduced modulo Lq (exact lattice phases, as in phase_table)
            auto one_dim = [&](const std::vector<int> &v) {
                std::vector<double2> t((size_t)m->Lq * v.size());
                for (int u = 0; u < m->Lq; u++)
                    for (size_t j = 0; j < v.size(); j++) {
                        const long k = ((long)u * v[j]) % m->Lq;
                        const double a = 2.0 * M_PI * (double)((k + m->Lq) % m->Lq) / (double)m->Lq;
                        t[(size_t)u * v.size() + j] = make_double2(std::cos(a), std::sin(a));
                    }
                return t;
            };
            const std::vector<double2> py = one_dim(ry), px = one_dim(rx);
            CK(upload(&m->d_dft_tabs, tabs, m->stream), "upload Fourier tables");
            CK(upload(&m->d_dft_phy, py, m->stream), "upload Fourier tables");
            CK(upload(&m->d_dft_phx, px, m->stream), "upload Fourier tables");
            if (split) {
                std::vector<float2> py32(py.size()), px32(px.size());
                for (size_t i = 0; i < py.size(); i++) py32[i] = make_float2((float)py[i].x, (float)py[i].y);
                for (size_t i = 0; i < px.size(); i++) px32[i] = make_float2((float)px[i].x, (float)px[i].y);
                CK(upload(&m->d_dft_phy32, py32, m->stream), "upload Fourier tables");
                CK(upload(&m->d_dft_phx32, px32, m->stream), "upload Fourier tables");
            }
        }
    }
    // the Fourier transform uses e^{i u.R''} for the classes
    {
        const std::vector<double2> cph = phase_table(m->Lq, m->cls);
        CK(upload(&m->d_clsph, cph, m->stream), "upload phase table");
        if (split) {
            std::vector<float2> c32(cph.size());
            for (size_t i = 0; i < cph.size(); i++) c32[i] = make_float2((float)cph[i].x, (float)cph[i].y);
            CK(upload(&m->d_clsph32, c32, m->stream), "upload phase table");
            // e^{-2 pi i n / Lf} of the split loop kernel, with exact quarter-turn values
            std::vector<float2> lph(m->Lf);
            for (int n = 0; n < m->Lf; n++) {
                const double a = 2.0 * M_PI * (double)n / (double)m->Lf;
                double c = std::cos(a), sn = std::sin(a);
                if ((4 * n) % m->Lf == 0) {
                    const int quarter = (4 * n) / m->Lf;
                    c = quarter == 0 ? 1.0 : quarter == 2 ? -1.0 : 0.0;
                    sn = quarter == 1 ? 1.0 : quarter == 3 ? -1.0 : 0.0;
                }
                lph[n] = make_float2((float)c, (float)-sn);
            }
            CK(upload(&m->d_lph32, lph, m->stream), "upload phase table");
        }
    }
    CK(dalloc(&m->d_E, Nk * ns), "cudaMalloc eigenvalues");
    CK(dalloc(&m->d_U, Nk * ns2), "cudaMalloc eigenvectors");
    CK(dalloc(&m->d_ft, Nk * ns), "cudaMalloc Fermi table");
    if (split) {
        CK(dalloc(&m->d_U32, Nk * ns2), "cudaMalloc eigenvectors");
        CK(dalloc(&m->d_ft32, Nk * ns), "cudaMalloc Fermi table");
        CK(dalloc(&m->d_Lc32, 2 * (size_t)m->Nq * m->nd * ns4), "cudaMalloc loops");
        CK(dalloc(&m->d_A32, 2 * (size_t)m->Nq * M2), "cudaMalloc projections");
        CK(dalloc(&m->d_X32, 2 * (size_t)m->Nq * M2), "cudaMalloc state copy");
    }
    CK(dalloc(&m->d_Lc, 2 * (size_t)m->Nq * m->nd * ns4), "cudaMalloc loops");
    int ndyh = 0;
    for (int v : m->dys) ndyh += v >= 0;
    // partial sums of both channels (the split two-band path sums P and C before one reduction)
    m->part_bytes = 2 * (size_t)m->Nq * max_partials * m->dxs.size() * ndyh * ns4 * (split ? sizeof(float2) : sizeof(double2));
    if (ns != 2) {
        if (!loops_gen_supported(m)) return fail(m, TUFRG_ENOTSUP, "bond set too large for the multi-orbital loop kernel");
        m->loops_tc = d.loops != TUFRG_LOOPS_SIMT && loops_tc_supported(m);
        m->gen_chunks = m->loops_tc ? 1 : plan_gen_chunks(m);
        // accumulators of one channel: one slot per (kx range, directly summed momentum), plus the FP64
        // range sums of the representatives under symmetry
        m->part_bytes = gen_part_bytes(m);
        if (m->loops_tc)
            CK(cudaMalloc(reinterpret_cast<void **>(&m->d_loop_w), loops_tc_w_bytes(m)), "cudaMalloc loop column sums");
    }
    m->products = split ? (d.products == TUFRG_PRODUCTS_AUTO ? TUFRG_PRODUCTS_TC : d.products) : TUFRG_PRODUCTS_SIMT;
    // product scratch: the large-M CUDA-core GEMMs' intermediate, or the tensor-core products' first product of both
    // channels (FP32 complex, the same bytes)
    if (m->M > 64 || split)
        CK(cudaMalloc(reinterpret_cast<void **>(&m->d_T), (size_t)m->Nq * M2 * sizeof(double2)), "cudaMalloc product scratch");
    CK(dalloc(&m->d_err, 1), "cudaMalloc error flag");
    CK(dalloc(&m->d_scal, 2), "cudaMalloc scalars");
    CK(cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream), "zero error flag");
    CK(cudaMalloc(&m->d_part, m->part_bytes), "cudaMalloc loop partials");
    CK(dalloc(&m->d_Xr, 2 * (size_t)m->ncls * M2), "cudaMalloc Fourier transforms");
    // partial sums of the sliced direct transform, or Z(u_x, R_y) of the separable one ([2][Lq][n_Ry][M^2])
    const size_t dft_scratch = m->dft_warps > 0 ? 2 * (size_t)m->Lq * m->dft_nry * M2
                                                : (size_t)m->dft_nsplit * 2 * m->ncls * M2;
    CK(cudaMalloc(&m->d_dftpart, dft_scratch * (split ? sizeof(float2) : sizeof(double2))),
       "cudaMalloc Fourier partials");
    if (split) CK(dalloc(&m->d_Xr32, 2 * (size_t)m->ncls * M2), "cudaMalloc Fourier transforms");
    if (loops2_supported(m)) CK(dalloc(&m->d_rec, Nk * 3), "cudaMalloc loop records");
    if (!split) CK(dalloc(&m->d_A, 2 * (size_t)m->Nq * M2), "cudaMalloc projections");   // split: FP32 copy only
    CK(dalloc(&m->d_amax, 4), "cudaMalloc reductions");
    CK(dalloc(&m->d_red, 512), "cudaMalloc reductions");

    // ---- eigensystem and chemical potential
    CK(launch_bands(m), "eigensolve");
    if (d.filling > 0) {
        std::vector<double> E(Nk * ns);
        CK(cudaMemcpyAsync(E.data(), m->d_E, sizeof(double) * E.size(), cudaMemcpyDeviceToHost, m->stream), "copy bands");
        CK(cudaStreamSynchronize(m->stream), "sync");
        double lo = *std::min_element(E.begin(), E.end()) - 1.0, hi = *std::max_element(E.begin(), E.end()) + 1.0;
        for (int it = 0; it < 200; it++) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            double n = 0.0;
            CK(launch_density(m, mid, d.T_mu, &n), "density");
            if (n < d.filling) lo = mid; else hi = mid;
        }
        m->mu = 0.5 * (lo + hi);
    } else {
        m->mu = d.mu;
    }
    // band basis: the bare vertex's projections transformed with the eigenvectors, then unit eigenvectors for the
    // band-diagonal loops (before the loop records, which hold projectors)
    if (m->basis == TUFRG_BASIS_BAND) CK(setup_band_flow(m), "band-basis set-up");
    if (loops2_supported(m)) CK(launch_loop_records_static(m), "loop records");
    if (m->regulator == TUFRG_REG_MOMENTUM_SHELL) {
        // the Fermi data of the momentum-shell loops do not depend on the flow scale: written once
        if (loops2_supported(m)) CK(launch_loop_records_shell(m), "loop records");
        else CK(launch_fermi_shell(m), "Fermi tables");
    }
    CK(cudaStreamSynchronize(m->stream), "init sync");
    TuneResult cached{};
    if (m->plan_cand.size() > 1 && tune_lookup(m, 3, &cached)) {
        m->plan = m->plan_cand[cached.choice];
        m->plan_ms = cached.cand_ms;
    } else if (m->plan_cand.size() > 1) {
        // autotune the loop k-sum's launch shape (ky ranges per column: grid depth against the per-column flush) on
        // this model's mesh; the P channel at T = 1 (the cost does not depend on the values)
        CK(launch_set_scalars(m, 1.0, 1.0), "set scalars");
        CK(launch_fermi(m), "loop records");
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        m->plan_ms.assign(m->plan_cand.size(), 0.0);
        int best = 0;
        for (size_t c = 0; c < m->plan_cand.size(); c++) {
            m->plan = m->plan_cand[c];
            CK(launch_loops2(m, 0), "loop autotune warm-up");
            CK(cudaEventRecord(e0, m->stream), "event");
            const int reps = 3;
            for (int r = 0; r < reps; r++) CK(launch_loops2(m, 0), "loop autotune");
            CK(cudaEventRecord(e1, m->stream), "event");
            CK(cudaEventSynchronize(e1), "event");
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1), "event");
            m->plan_ms[c] = ms / reps;
            if (m->plan_ms[c] < m->plan_ms[best]) best = (int)c;
        }
        m->plan = m->plan_cand[best];
        TuneResult r{};
        r.choice = best;
        r.cand_ms = m->plan_ms;
        tune_store(m, 3, r);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        m->launches = 0;
        m->loop_launches = 0;
        int dev_err = 0;
        CK(cudaMemcpy(&dev_err, m->d_err, sizeof(int), cudaMemcpyDeviceToHost), "copy error flag");
        if (dev_err) return fail(m, TUFRG_ETIMEOUT, "a bounded device-side wait gave up during autotuning");
    }
    if (split && d.products == TUFRG_PRODUCTS_AUTO && tune_lookup(m, 0, &cached)) {
        m->products = cached.choice;
        m->tune_ms[0] = cached.ms[0];
        m->tune_ms[1] = cached.ms[1];
        m->tc_tile_ms = cached.cand_ms;
        m->tc_ntiles = cached.aux;
    } else if (split && d.products == TUFRG_PRODUCTS_AUTO) {
        // autotune the products backend on this model's sizes (the cost does not depend on the values)
        const size_t nA = 2 * (size_t)m->Nq * M2;
        double2 *tmp = nullptr;
        CK(dalloc(&tmp, nA), "cudaMalloc autotune output");
        CK(cudaMemsetAsync(m->d_A32, 0, sizeof(float2) * nA, m->stream), "zero");
        CK(cudaMemsetAsync(m->d_Lc32, 0, sizeof(float2) * 2 * (size_t)m->Nq * m->nd * ns4, m->stream), "zero");
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        const int cand[2] = {TUFRG_PRODUCTS_TC, TUFRG_PRODUCTS_SIMT};
        CK(launch_set_scalars(m, 1.0, 1.0), "set scalars");
        // the tensor cores at each column-tile count (tile width), then the CUDA cores
        const std::vector<int> tiles = tc_tile_candidates(m);
        m->tc_tile_ms.assign(tiles.size(), 0.0);
        int best_tiles = tiles[0];
        for (int c = 0; c < 2; c++) {
            m->products = cand[c];
            for (size_t t = 0; t < (c == 0 ? tiles.size() : 1); t++) {
                if (c == 0) m->tc_ntiles = tiles[t];
                CK(launch_vlv(m, m->d_A, 3, tmp), "autotune warm-up");
                CK(cudaEventRecord(e0, m->stream), "event");
                const int reps = 3;
                for (int r = 0; r < reps; r++) CK(launch_vlv(m, m->d_A, 3, tmp), "autotune");
                CK(cudaEventRecord(e1, m->stream), "event");
                CK(cudaEventSynchronize(e1), "event");
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1), "event");
                if (c == 0) {
                    m->tc_tile_ms[t] = ms / reps;
                    if (t == 0 || m->tc_tile_ms[t] < m->tune_ms[0]) {
                        m->tune_ms[0] = m->tc_tile_ms[t];
                        best_tiles = tiles[t];
                    }
                } else {
                    m->tune_ms[1] = ms / reps;
                }
            }
        }
        m->tc_ntiles = best_tiles;
        m->products = m->tune_ms[0] <= m->tune_ms[1] ? TUFRG_PRODUCTS_TC : TUFRG_PRODUCTS_SIMT;
        TuneResult r{{m->tune_ms[0], m->tune_ms[1]}, m->products};
        r.cand_ms = m->tc_tile_ms;
        r.aux = m->tc_ntiles;
        tune_store(m, 0, r);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(tmp);
        m->launches = 0;
        m->loop_launches = 0;
        int dev_err = 0;
        CK(cudaMemcpy(&dev_err, m->d_err, sizeof(int), cudaMemcpyDeviceToHost), "copy error flag");
        if (dev_err) return fail(m, TUFRG_ETIMEOUT, "a bounded device-side wait gave up during autotuning");
    }
    if (m->sym_state && tune_lookup(m, 1 + m->products, &cached)) {
        m->sym_tune_ms[0] = cached.ms[0];
        m->sym_tune_ms[1] = cached.ms[1];
    } else if (m->sym_state) {
        // symmetric states: projections and products for the orbit representatives plus the gather of the
        // other momenta, against both for every momentum (on zeroed operands: the cost does not depend on
        // the values).  Reported only: the representatives' path is taken whenever the symmetries hold (a
        // timing-based choice would differ between processes, e.g. under a profiler)
        const size_t nA = 2 * (size_t)m->Nq * M2;
        double2 *tmp = nullptr;
        CK(dalloc(&tmp, nA), "cudaMalloc autotune output");
        CK(cudaMemsetAsync(tmp, 0, sizeof(double2) * nA, m->stream), "zero");
        if (split) {
            CK(cudaMemsetAsync(m->d_A32, 0, sizeof(float2) * nA, m->stream), "zero");
            CK(cudaMemsetAsync(m->d_X32, 0, sizeof(float2) * nA, m->stream), "zero");
            CK(cudaMemsetAsync(m->d_Xr32, 0, sizeof(float2) * 2 * (size_t)m->ncls * M2, m->stream), "zero");
            CK(cudaMemsetAsync(m->d_Lc32, 0, sizeof(float2) * 2 * (size_t)m->Nq * m->nd * ns4, m->stream), "zero");
        } else {
            CK(cudaMemsetAsync(m->d_A, 0, sizeof(double2) * nA, m->stream), "zero");
            CK(cudaMemsetAsync(m->d_Xr, 0, sizeof(double2) * 2 * (size_t)m->ncls * M2, m->stream), "zero");
            CK(cudaMemsetAsync(m->d_Lc, 0, sizeof(double2) * 2 * (size_t)m->Nq * m->nd * ns4, m->stream), "zero");
        }
        CK(launch_set_scalars(m, 1.0, 1.0), "set scalars");
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        for (int c = 0; c < 2; c++) {
            auto run = [&]() -> cudaError_t {
                // the FP64 path projects the (zero) state in tmp into d_A; the products then overwrite tmp
                const int *ql = c ? m->d_loop_list : nullptr;
                const int nl = c ? m->n_loop_q : 0;
                cudaError_t e = launch_project(m, tmp, split ? m->d_X32 : nullptr, 3, split ? nullptr : m->d_A, ql, nl);
                if (e == cudaSuccess) e = c ? launch_products_sym(m, 3, tmp) : launch_vlv(m, m->d_A, 3, tmp);
                return e;
            };
            CK(run(), "symmetric-state autotune warm-up");
            CK(cudaEventRecord(e0, m->stream), "event");
            const int reps = 3;
            for (int r = 0; r < reps; r++) CK(run(), "symmetric-state autotune");
            CK(cudaEventRecord(e1, m->stream), "event");
            CK(cudaEventSynchronize(e1), "event");
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1), "event");
            m->sym_tune_ms[c] = ms / reps;
        }
        tune_store(m, 1 + m->products, TuneResult{{m->sym_tune_ms[0], m->sym_tune_ms[1]}, 1});
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(tmp);
        m->launches = 0;
        m->loop_launches = 0;
        int dev_err = 0;
        CK(cudaMemcpy(&dev_err, m->d_err, sizeof(int), cudaMemcpyDeviceToHost), "copy error flag");
        if (dev_err) return fail(m, TUFRG_ETIMEOUT, "a bounded device-side wait gave up during autotuning");
    }
    return TUFRG_OK;
} catch (const std::exception &ex) {
    return host_alloc_fail(out ? *out : nullptr, ex);
}

tufrg_status tufrg_model_info(const tufrg_model *m, int *products, double *ms_tc, double *ms_simt)
{
    if (!m) return TUFRG_EINVAL;
    if (products) *products = m->products;
    if (ms_tc) *ms_tc = m->tune_ms[0];
    if (ms_simt) *ms_simt = m->tune_ms[1];
    return TUFRG_OK;
}

tufrg_status tufrg_loop_momenta(const tufrg_model *m, int *n_direct)
{
    if (!m || !n_direct) return TUFRG_EINVAL;
    *n_direct = m->n_loop_q;
    return TUFRG_OK;
}

tufrg_status tufrg_loops_info(const tufrg_model *m, int *backend)
{
    if (!m || !backend) return TUFRG_EINVAL;
    *backend = m->loops_tc ? TUFRG_LOOPS_TC : TUFRG_LOOPS_SIMT;
    return TUFRG_OK;
}

tufrg_status tufrg_products_tiles(const tufrg_model *m, int *tile_width, int *n_candidates, double *h_ms, int n_ms)
{
    if (!m || !tile_width || !n_candidates || (n_ms > 0 && !h_ms) || n_ms < 0) return TUFRG_EINVAL;
    *tile_width = (m->precision != TUFRG_FP64) ? tc_tile_width(m) : 0;
    *n_candidates = (int)m->tc_tile_ms.size();
    for (int i = 0; i < n_ms && i < (int)m->tc_tile_ms.size(); i++) h_ms[i] = m->tc_tile_ms[i];
    return TUFRG_OK;
}

tufrg_status tufrg_loop_tiles(const tufrg_model *m, int *ky_chunks, int *n_candidates, double *h_ms, int n_ms)
{
    if (!m || !ky_chunks || !n_candidates || (n_ms > 0 && !h_ms) || n_ms < 0) return TUFRG_EINVAL;
    *ky_chunks = m->plan.ky_chunks;
    *n_candidates = (int)m->plan_ms.size();
    for (int i = 0; i < n_ms && i < (int)m->plan_ms.size(); i++) h_ms[i] = m->plan_ms[i];
    return TUFRG_OK;
}

tufrg_status tufrg_band_basis(tufrg_model *m, const void *d_state, void *d_out)
{
    if (!m || !d_state || !d_out) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!band_basis_supported(m))
        return fail(m, TUFRG_ENOTSUP, "the band-basis transformation supports two-band models with M <= 64");
    CK(launch_band_basis(m, reinterpret_cast<const double2 *>(d_state), reinterpret_cast<double2 *>(d_out)),
       "band-basis transformation");
    return TUFRG_OK;
}

tufrg_status tufrg_round_f32(const void *d_in, void *d_out, size_t n, void *cuda_stream)
{
    if (n > 0 && (!d_in || !d_out)) return TUFRG_EINVAL;
    const cudaError_t e = launch_round_f32(static_cast<const double *>(d_in), static_cast<float *>(d_out), n,
                                           static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? TUFRG_OK : TUFRG_ECUDA;
}

tufrg_status tufrg_widen_f64(const void *d_in, void *d_out, size_t n, void *cuda_stream)
{
    if (n > 0 && (!d_in || !d_out)) return TUFRG_EINVAL;
    const cudaError_t e = launch_widen_f64(static_cast<const float *>(d_in), static_cast<double *>(d_out), n,
                                           static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? TUFRG_OK : TUFRG_ECUDA;
}

tufrg_status tufrg_symmetry_info(const tufrg_model *m, int *in_use, double *ms_general, double *ms_reps)
{
    if (!m || !in_use || !ms_general || !ms_reps) return TUFRG_EINVAL;
    *in_use = m->sym_state ? 1 : 0;
    *ms_general = m->sym_state ? m->sym_tune_ms[0] : -1.0;
    *ms_reps = m->sym_state ? m->sym_tune_ms[1] : -1.0;
    return TUFRG_OK;
}

void tufrg_free(tufrg_model *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    release(m);
    delete m;
}

const char *tufrg_last_error(const tufrg_model *m)
{
    return m ? m->err.c_str() : "model handle is NULL";
}

tufrg_status tufrg_dims(const tufrg_model *m, int *Nq, int *M, int *n_delta, int *Nk, double *mu)
{
    if (!m) return TUFRG_EINVAL;
    if (Nq) *Nq = m->Nq;
    if (M) *M = m->M;
    if (n_delta) *n_delta = m->nd;
    if (Nk) *Nk = m->Nk;
    if (mu) *mu = m->mu;
    return TUFRG_OK;
}

tufrg_status tufrg_deltas(const tufrg_model *m, int *h_out)
{
    if (!m || !h_out) return TUFRG_EINVAL;
    std::memcpy(h_out, m->deltas.data(), sizeof(int) * m->deltas.size());
    return TUFRG_OK;
}

tufrg_status tufrg_gather_table(const tufrg_model *m, int channel, int *h_out, int cap, int *n_terms)
{
    if (!m || channel < 0 || channel > 1 || !n_terms || cap < 0) return TUFRG_EINVAL;
    const int n = (int)m->gtab_export[channel].size() / 9;
    *n_terms = n;
    if (h_out) std::memcpy(h_out, m->gtab_export[channel].data(), sizeof(int) * 9 * (size_t)std::min(n, cap));
    return TUFRG_OK;
}

tufrg_status tufrg_bands(tufrg_model *m, double *d_E, double *d_U)
{
    if (!m || !d_E || !d_U) return fail(m, TUFRG_EINVAL, "NULL argument");
    CK(cudaMemcpyAsync(d_E, m->d_E, sizeof(double) * m->Nk * m->ns, cudaMemcpyDeviceToDevice, m->stream), "copy bands");
    CK(cudaMemcpyAsync(d_U, m->d_U, sizeof(double2) * m->Nk * m->ns * m->ns, cudaMemcpyDeviceToDevice, m->stream), "copy bands");
    return TUFRG_OK;
}

tufrg_status tufrg_loops(tufrg_model *m, double T, int channel_mask, void *d_loops)
{
    if (!m || !d_loops) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!(T > 0) || !std::isfinite(T)) return fail(m, TUFRG_EINVAL, "T must be positive and finite");
    if (channel_mask & ~3) return fail(m, TUFRG_EINVAL, "channel_mask must be a subset of P|C");
    CK(launch_set_scalars(m, T, 1.0), "set temperature");
    CK(surrogate_rearm(m), "re-arm surrogate");
    CK(launch_fermi(m), "fermi tables");
    CK(launch_loops(m, channel_mask), "loop k-sum");
    const size_t per = (size_t)m->Nq * m->nd * m->ns * m->ns * m->ns * m->ns;
    for (int ch = 0; ch < 2; ch++)
        if ((channel_mask >> ch) & 1)
            CK(cudaMemcpyAsync(reinterpret_cast<double2 *>(d_loops) + ch * per, m->d_Lc + ch * per, sizeof(double2) * per,
                               cudaMemcpyDeviceToDevice, m->stream), "copy loops");
    return TUFRG_OK;
}

tufrg_status tufrg_project(tufrg_model *m, const void *d_state, int channel_mask, void *d_Ahat, double *h_amax)
{
    if (!m || !d_state || !d_Ahat) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (channel_mask & ~3) return fail(m, TUFRG_EINVAL, "channel_mask must be a subset of P|C");
    const double2 *st = reinterpret_cast<const double2 *>(d_state);
    const float2 *st32 = nullptr;
    if (m->precision != TUFRG_FP64 && m->dft_warps == 0) {
        CK(launch_to_f32(m, st, m->d_X32, state_elems(m)), "state conversion");
        st32 = m->d_X32;
    }
    CK(launch_dft(m, st, st32, channel_mask), "Fourier transform");
    if (m->precision != TUFRG_FP64 && !st32) st32 = m->d_X32;   // written by the separable transform
    CK(launch_project(m, st, st32, channel_mask, reinterpret_cast<double2 *>(d_Ahat)), "projections");
    if (h_amax) {
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, m->d_amax, sizeof(bits), cudaMemcpyDeviceToHost, m->stream), "copy max");
        CK(cudaStreamSynchronize(m->stream), "sync");
        std::memcpy(h_amax, &bits, sizeof(double));
    }
    return TUFRG_OK;
}

tufrg_status tufrg_rhs(tufrg_model *m, double T, const void *d_state, int channel_mask, void *d_dstate)
try {
    if (!m || !d_state || !d_dstate) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!(T > 0) || !std::isfinite(T)) return fail(m, TUFRG_EINVAL, "T must be positive and finite");
    if (channel_mask & ~(3 | TUFRG_SYMMETRIC_STATE))
        return fail(m, TUFRG_EINVAL, "channel_mask must be a subset of P|C, optionally with TUFRG_SYMMETRIC_STATE");
    CK(launch_set_scalars(m, T, 1.0), "set temperature");
    CK(surrogate_rearm(m), "re-arm surrogate");
    auto direct = [&]() {
        return rhs_device(m, reinterpret_cast<const double2 *>(d_state), channel_mask & 3,
                          reinterpret_cast<double2 *>(d_dstate), nullptr, (channel_mask & TUFRG_SYMMETRIC_STATE) != 0);
    };
    // The launches after the temperature (which they read from device memory) are replayed from a captured graph:
    // the same kernels in the same order without the gaps between launches.  Direct launches instead while the
    // phases are being timed, with a loop surrogate, or when the caller is capturing the stream itself.  The legacy
    // default stream cannot be captured: there the graph runs on a private stream joined to it by events.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (m->timing || m->sur || m->rhs_graph_off ||
        (m->stream != nullptr && (cudaStreamIsCapturing(m->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)))
        return direct();
    tufrg_model::RhsGraph *g = nullptr;
    for (auto &r : m->rhs_graphs)
        if (r.in == d_state && r.out == d_dstate && r.mask == channel_mask) g = &r;
    auto make_room = [&]() {   // the least recently used entry makes room (at most 4 kept)
        if (m->rhs_graphs.size() < 4) return;
        auto lru = m->rhs_graphs.begin();
        for (auto it = m->rhs_graphs.begin(); it != m->rhs_graphs.end(); ++it)
            if (it->used < lru->used) lru = it;
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        m->rhs_graphs.erase(lru);
    };
    if (!g) {
        // first use of these buffers: launch directly and remember them (a one-off call costs no capture)
        make_room();
        m->rhs_graphs.push_back(tufrg_model::RhsGraph{d_state, d_dstate, channel_mask, nullptr, 0, 0, ++m->rhs_graph_clock});
        return direct();
    }
    // on the legacy default stream: the private stream, ordered after it here and before it at the end
    const cudaStream_t user = m->stream;
    if (user == nullptr) {
        if (!m->rhs_stream) {
            CK(cudaStreamCreateWithFlags(&m->rhs_stream, cudaStreamNonBlocking), "create stream");
            CK(cudaEventCreateWithFlags(&m->rhs_ev[0], cudaEventDisableTiming), "create event");
            CK(cudaEventCreateWithFlags(&m->rhs_ev[1], cudaEventDisableTiming), "create event");
        }
        CK(cudaEventRecord(m->rhs_ev[0], user), "record");
        CK(cudaStreamWaitEvent(m->rhs_stream, m->rhs_ev[0], 0), "wait");
        m->stream = m->rhs_stream;
    }
    struct Rejoin {   // back to the caller's stream on every return
        tufrg_model *m;
        cudaStream_t user;
        ~Rejoin()
        {
            if (user != nullptr || m->stream == nullptr) return;
            cudaEventRecord(m->rhs_ev[1], m->stream);
            cudaStreamWaitEvent(user, m->rhs_ev[1], 0);
            m->stream = user;
        }
    } rejoin{m, user};
    if (!g->exec) {
        const long long l0 = m->launches, ll0 = m->loop_launches;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const tufrg_status st = direct();
        const cudaError_t ce = cudaStreamEndCapture(m->stream, &graph);
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = (st == TUFRG_OK && ce == cudaSuccess) ? cudaGraphInstantiate(&exec, graph, 0) : cudaErrorUnknown;
        if (graph) cudaGraphDestroy(graph);
        const long long dl = m->launches - l0, dll = m->loop_launches - ll0;
        m->launches = l0;
        m->loop_launches = ll0;
        if (st != TUFRG_OK) return st;
        if (ce != cudaSuccess || ie != cudaSuccess) {
            // not capturable here: launch directly from now on
            (void)cudaGetLastError();
            m->rhs_graph_off = true;
            return direct();
        }
        g->exec = exec;
        g->launches = dl;
        g->loop_launches = dll;
    }
    g->used = ++m->rhs_graph_clock;
    CK(cudaGraphLaunch(g->exec, m->stream), "right-hand side graph");
    m->launches += g->launches;
    m->loop_launches += g->loop_launches;
    return TUFRG_OK;
} catch (const std::exception &ex) {
    return host_alloc_fail(m, ex);
}

// ------------------------------------------------------------------ right-hand side over shards of momenta

namespace {
// checks a shard's momentum list (distinct momenta in [0, Nq)) and uploads it to the model's list buffer
tufrg_status upload_shard(tufrg_model *m, int n_q, const int *h_q_list)
{
    if (n_q < 1 || n_q > m->Nq || !h_q_list) return fail(m, TUFRG_EINVAL, "the shard needs 1 to Nq momenta");
    std::vector<char> seen(m->Nq, 0);
    for (int i = 0; i < n_q; i++) {
        const int q = h_q_list[i];
        if (q < 0 || q >= m->Nq || seen[q]) return fail(m, TUFRG_EINVAL, "shard momenta must be distinct and in [0, Nq)");
        seen[q] = 1;
    }
    if (m->sur) return fail(m, TUFRG_ENOTSUP, "the sharded right-hand side does not use the loop surrogate: detach it");
    if (!m->d_shard_q) CK(dalloc(&m->d_shard_q, m->Nq), "cudaMalloc shard list");
    CK(cudaMemcpyAsync(m->d_shard_q, h_q_list, sizeof(int) * n_q, cudaMemcpyHostToDevice, m->stream), "upload shard list");
    return TUFRG_OK;
}
}  // namespace

tufrg_status tufrg_form_factors(const tufrg_model *m, double *h_W, int *h_labels)
{
    if (!m || !h_W || !h_labels) return TUFRG_EINVAL;
    if (m->ffW.empty()) return TUFRG_ENOTSUP;
    std::copy(m->ffW.begin(), m->ffW.end(), h_W);
    std::copy(m->ff_labels.begin(), m->ff_labels.end(), h_labels);
    return TUFRG_OK;
}

tufrg_status tufrg_irrep_basis(tufrg_model *m, const void *d_state, int inverse, void *d_out)
{
    if (!m || !d_state || !d_out) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (m->ffW.empty()) return fail(m, TUFRG_ENOTSUP, "the bond set is not closed under the point group");
    if (d_state == d_out) return fail(m, TUFRG_EINVAL, "the transformation does not work in place");
    CK(launch_irrep_basis(m, reinterpret_cast<const double2 *>(d_state), inverse ? 1 : 0, reinterpret_cast<double2 *>(d_out)),
       "irrep form factors");
    return TUFRG_OK;
}

tufrg_status tufrg_shard_classes(const tufrg_model *m, int *ncls, int *h_cls)
{
    if (!m || !ncls) return TUFRG_EINVAL;
    *ncls = m->ncls;
    if (h_cls) std::copy(m->cls.begin(), m->cls.end(), h_cls);
    return TUFRG_OK;
}

tufrg_status tufrg_rhs_shard_transform(tufrg_model *m, const void *d_state_local, int n_q, const int *h_q_list,
                                       int channel_mask, void *d_xr)
try {
    if (!m || !d_state_local || !d_xr) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (channel_mask & ~3) return fail(m, TUFRG_EINVAL, "channel_mask must be a subset of P|C");
    tufrg_status st = upload_shard(m, n_q, h_q_list);
    if (st != TUFRG_OK) return st;
    CK(launch_shard_dft(m, reinterpret_cast<const double2 *>(d_state_local), n_q, m->d_shard_q, channel_mask,
                        reinterpret_cast<double2 *>(d_xr)), "shard Fourier transform");
    return TUFRG_OK;
} catch (const std::exception &ex) {
    return host_alloc_fail(m, ex);
}

tufrg_status tufrg_rhs_shard_finish(tufrg_model *m, double T, const void *d_state_local, int n_q, const int *h_q_list,
                                    const void *d_xr, int channel_mask, void *d_dstate_local)
try {
    if (!m || !d_state_local || !d_xr || !d_dstate_local) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!(T > 0) || !std::isfinite(T)) return fail(m, TUFRG_EINVAL, "T must be positive and finite");
    if (channel_mask & ~3) return fail(m, TUFRG_EINVAL, "channel_mask must be a subset of P|C");
    tufrg_status st = upload_shard(m, n_q, h_q_list);
    if (st != TUFRG_OK) return st;
    const bool split = m->precision != TUFRG_FP64;
    const size_t M2 = (size_t)m->M * m->M, nx = 2 * (size_t)m->ncls * M2;
    const double2 *xr = reinterpret_cast<const double2 *>(d_xr);
    const double2 *X = reinterpret_cast<const double2 *>(d_state_local);
    // the summed transforms in the model's working precision
    if (split) CK(launch_to_f32(m, xr, m->d_Xr32, nx), "transform conversion");
    else CK(cudaMemcpyAsync(m->d_Xr, xr, sizeof(double2) * nx, cudaMemcpyDeviceToDevice, m->stream), "copy transforms");
    CK(launch_set_scalars(m, T, 1.0), "set temperature");
    CK(launch_fermi(m), "fermi tables");
    CK(launch_loops_list(m, channel_mask, m->d_shard_q, n_q), "loop k-sum of the shard");
    // the shard's rows in FP32 for the split path (list order, in the front of the model's copy)
    if (split) CK(launch_to_f32(m, X, m->d_X32, 2 * (size_t)n_q * M2), "state conversion");
    CK(launch_project_local(m, X, split ? m->d_X32 : nullptr, channel_mask, split ? nullptr : m->d_A, m->d_shard_q, n_q),
       "projections of the shard");
    if (!m->d_shard_out) CK(dalloc(&m->d_shard_out, state_elems(m)), "cudaMalloc shard products");
    CK(launch_vlv(m, m->d_A, channel_mask, m->d_shard_out, m->d_shard_q, n_q), "V.L.V products of the shard");
    CK(launch_shard_gather(m, m->d_shard_out, n_q, m->d_shard_q, reinterpret_cast<double2 *>(d_dstate_local)),
       "gather of the shard's rows");
    return TUFRG_OK;
} catch (const std::exception &ex) {
    return host_alloc_fail(m, ex);
}

tufrg_status tufrg_rhs_host(tufrg_model *m, double T, const void *h_state, int channel_mask, void *h_dstate)
{
    if (!m || !h_state || !h_dstate) return fail(m, TUFRG_EINVAL, "NULL argument");
    const size_t bytes = sizeof(double2) * state_elems(m);
    if (!m->d_state_in) {
        CK(cudaMalloc(&m->d_state_in, bytes), "cudaMalloc state");
        CK(cudaMalloc(&m->d_state_out, bytes), "cudaMalloc state");
    }
    CK(cudaMemcpyAsync(m->d_state_in, h_state, bytes, cudaMemcpyHostToDevice, m->stream), "copy state in");
    tufrg_status st = tufrg_rhs(m, T, m->d_state_in, channel_mask, m->d_state_out);
    if (st != TUFRG_OK) return st;
    CK(cudaMemcpyAsync(h_dstate, m->d_state_out, bytes, cudaMemcpyDeviceToHost, m->stream), "copy derivative out");
    int dev_err = 0;
    CK(cudaMemcpyAsync(&dev_err, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream), "copy error flag");
    CK(cudaStreamSynchronize(m->stream), "sync");
    if (dev_err) return fail(m, TUFRG_ETIMEOUT, "a bounded device-side wait gave up");
    return TUFRG_OK;
}

tufrg_status tufrg_rhs_host_batch(tufrg_model *m, int n, const double *T, const void *const *h_states, int channel_mask,
                                  void *const *h_dstates)
{
    if (!m) return TUFRG_EINVAL;
    if (n < 0 || (n > 0 && (!T || !h_states || !h_dstates))) return fail(m, TUFRG_EINVAL, "bad batch arguments");
    if (channel_mask & ~(3 | TUFRG_SYMMETRIC_STATE))
        return fail(m, TUFRG_EINVAL, "channel_mask must be a subset of P|C, optionally with TUFRG_SYMMETRIC_STATE");
    for (int i = 0; i < n; i++) {
        if (!(T[i] > 0) || !std::isfinite(T[i])) return fail(m, TUFRG_EINVAL, "T must be positive and finite");
        if (!h_states[i] || !h_dstates[i]) return fail(m, TUFRG_EINVAL, "NULL host buffer");
    }
    if (n == 0) return TUFRG_OK;
    const size_t bytes = sizeof(double2) * state_elems(m);
    if (!m->d_bin[0]) {
        for (int b = 0; b < 2; b++) {
            CK(cudaMalloc(&m->d_bin[b], bytes), "cudaMalloc state");
            CK(cudaMalloc(&m->d_bout[b], bytes), "cudaMalloc state");
            CK(cudaEventCreateWithFlags(&m->ev_in[b], cudaEventDisableTiming), "event");
            CK(cudaEventCreateWithFlags(&m->ev_comp[b], cudaEventDisableTiming), "event");
            CK(cudaEventCreateWithFlags(&m->ev_out[b], cudaEventDisableTiming), "event");
        }
        CK(cudaStreamCreateWithFlags(&m->s_h2d, cudaStreamNonBlocking), "stream");
        CK(cudaStreamCreateWithFlags(&m->s_d2h, cudaStreamNonBlocking), "stream");
    }
    // step i uses buffer pair b = i mod 2: its input copy waits until step i - 2 has been evaluated, its
    // evaluation until the input has arrived and step i - 2's output has left, its output copy until it
    // has been evaluated
    tufrg_status st = TUFRG_OK;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && st == TUFRG_OK && e == cudaSuccess; i++) {
        const int b = i & 1;
        if (i >= 2) e = cudaStreamWaitEvent(m->s_h2d, m->ev_comp[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_bin[b], h_states[i], bytes, cudaMemcpyHostToDevice, m->s_h2d);
        if (e == cudaSuccess) e = cudaEventRecord(m->ev_in[b], m->s_h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->stream, m->ev_in[b], 0);
        if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(m->stream, m->ev_out[b], 0);
        if (e != cudaSuccess) break;
        st = tufrg_rhs(m, T[i], m->d_bin[b], channel_mask, m->d_bout[b]);
        if (st != TUFRG_OK) break;
        e = cudaEventRecord(m->ev_comp[b], m->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->s_d2h, m->ev_comp[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_dstates[i], m->d_bout[b], bytes, cudaMemcpyDeviceToHost, m->s_d2h);
        if (e == cudaSuccess) e = cudaEventRecord(m->ev_out[b], m->s_d2h);
    }
    // the host buffers stay in use until every queued copy has finished, also after an error
    const cudaError_t e1 = cudaStreamSynchronize(m->s_h2d), e2 = cudaStreamSynchronize(m->stream),
                      e3 = cudaStreamSynchronize(m->s_d2h);
    if (st != TUFRG_OK) return st;
    if (e != cudaSuccess) return cuda_fail(m, e, "pipelined host-buffer evaluation");
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
        return cuda_fail(m, e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3, "pipelined host-buffer evaluation");
    return read_device_error(m);
}

tufrg_status tufrg_flow(tufrg_model *m, const tufrg_flow_opts *o, void *d_state_out, tufrg_flow_result *res)
{
    tufrg_status st = flow_check_args(m, o, res);
    if (st != TUFRG_OK) return st;
    if (m->flow_open) return fail(m, TUFRG_EINVAL, "a stepwise flow is open on this model");
    const auto t_start = std::chrono::steady_clock::now();
    std::memset(res, 0, sizeof(*res));
    cudaStream_t user;
    if ((st = flow_enter(m, &user)) != TUFRG_OK) return st;
    st = flow_prepare(m, o);
    // replay the captured attempt until the device controller stops the flow
    while (st == TUFRG_OK && m->h_flow->status == 0) {
        cudaError_t e = cudaGraphLaunch(m->step_graph, m->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_flow, m->d_flow, sizeof(FlowDev), cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) st = cuda_fail(m, e, "flow graph");
        else if (m->h_flow->status != 0) break;
    }
    if (st == TUFRG_OK) st = read_device_error(m);
    if (st == TUFRG_OK) st = flow_finish(m, d_state_out, res);
    const tufrg_status st2 = flow_leave(m, user);
    res->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    return st != TUFRG_OK ? st : st2;
}

// ---- the flow step by step, with checkpoints

tufrg_status tufrg_flow_start(tufrg_model *m, const tufrg_flow_opts *o)
{
    tufrg_flow_result unused{};
    tufrg_status st = flow_check_args(m, o, &unused);
    if (st != TUFRG_OK) return st;
    if (m->flow_open) return fail(m, TUFRG_EINVAL, "a stepwise flow is already open on this model");
    cudaStream_t user;
    if ((st = flow_enter(m, &user)) != TUFRG_OK) return st;
    st = flow_prepare(m, o);
    if (st != TUFRG_OK) {
        flow_leave(m, user);
        return st;
    }
    m->flow_open = true;
    m->flow_user = user;
    m->flow_mask = o->channel_mask;
    m->flow_t0 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
    return TUFRG_OK;
}

tufrg_status tufrg_flow_step(tufrg_model *m, tufrg_flow_step_info *s)
{
    if (!m || !s) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!m->flow_open) return fail(m, TUFRG_EINVAL, "no stepwise flow is open on this model");
    if (m->h_flow->status == 0) {
        cudaError_t e = cudaGraphLaunch(m->step_graph, m->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(m->h_flow, m->d_flow, sizeof(FlowDev), cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return cuda_fail(m, e, "flow graph");
    }
    const FlowDev &f = *m->h_flow;
    s->T = std::exp(f.x);
    s->h = f.h;
    s->err = f.err;
    s->amax = f.amax;
    s->n_steps = f.n_steps;
    s->n_reject = f.n_reject;
    s->accepted = f.accepted;
    s->status = f.status;
    return read_device_error(m);
}

tufrg_status tufrg_flow_amax_channels(tufrg_model *m, double *h_amax)
{
    if (!m || !h_amax) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!m->d_amax_ch) CK(cudaMalloc(reinterpret_cast<void **>(&m->d_amax_ch), 2 * sizeof(unsigned long long)), "cudaMalloc");
    CK(launch_amax_channels(m, m->sym_state), "max |A| per channel");
    unsigned long long b[2];
    CK(cudaMemcpyAsync(b, m->d_amax_ch, sizeof(b), cudaMemcpyDeviceToHost, m->stream), "copy maxima");
    CK(cudaStreamSynchronize(m->stream), "sync");
    for (int c = 0; c < 2; c++) h_amax[c] = bits_to_double(b[c]);
    return TUFRG_OK;
}

tufrg_status tufrg_flow_end(tufrg_model *m, void *d_state_out, tufrg_flow_result *res)
{
    if (!m || !res) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!m->flow_open) return fail(m, TUFRG_EINVAL, "no stepwise flow is open on this model");
    std::memset(res, 0, sizeof(*res));
    tufrg_status st = read_device_error(m);
    if (st == TUFRG_OK) st = flow_finish(m, d_state_out, res);
    const tufrg_status st2 = flow_leave(m, m->flow_user);
    m->flow_open = false;
    res->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count() - m->flow_t0;
    return st != TUFRG_OK ? st : st2;
}

size_t tufrg_flow_checkpoint_bytes(const tufrg_model *m)
{
    if (!m) return 0;
    return sizeof(CkptHeader) + sizeof(FlowDev) + 2 * sizeof(double2) * state_elems(m);
}

tufrg_status tufrg_flow_save(tufrg_model *m, void *h_buf, size_t bytes)
{
    if (!m || !h_buf) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (!m->flow_open) return fail(m, TUFRG_EINVAL, "no stepwise flow is open on this model");
    if (m->sur) return fail(m, TUFRG_ENOTSUP, "checkpoints of flows with a loop surrogate are not supported");
    if (bytes < tufrg_flow_checkpoint_bytes(m)) return fail(m, TUFRG_EINVAL, "checkpoint buffer too small");
    const size_t n = state_elems(m);
    CkptHeader h = ckpt_header(m, m->flow_mask);
    unsigned char *p = static_cast<unsigned char *>(h_buf);
    std::memcpy(p, &h, sizeof(h));
    CK(cudaMemcpyAsync(p + sizeof(h), m->d_flow, sizeof(FlowDev), cudaMemcpyDeviceToHost, m->stream), "copy controller");
    CK(cudaMemcpyAsync(p + sizeof(h) + sizeof(FlowDev), m->d_y, sizeof(double2) * n, cudaMemcpyDeviceToHost, m->stream),
       "copy state");
    CK(cudaMemcpyAsync(p + sizeof(h) + sizeof(FlowDev) + sizeof(double2) * n, m->d_k[0], sizeof(double2) * n,
                       cudaMemcpyDeviceToHost, m->stream), "copy derivative");
    CK(cudaStreamSynchronize(m->stream), "sync");
    return TUFRG_OK;
}

tufrg_status tufrg_flow_resume(tufrg_model *m, const tufrg_flow_opts *o, const void *h_buf, size_t bytes)
{
    tufrg_flow_result unused{};
    tufrg_status st = flow_check_args(m, o, &unused);
    if (st != TUFRG_OK) return st;
    if (!h_buf) return fail(m, TUFRG_EINVAL, "NULL argument");
    if (m->flow_open) return fail(m, TUFRG_EINVAL, "a stepwise flow is already open on this model");
    if (m->sur) return fail(m, TUFRG_ENOTSUP, "checkpoints of flows with a loop surrogate are not supported");
    if (bytes < tufrg_flow_checkpoint_bytes(m)) return fail(m, TUFRG_EINVAL, "checkpoint buffer too small");
    CkptHeader h;
    std::memcpy(&h, h_buf, sizeof(h));
    const CkptHeader want = ckpt_header(m, o->channel_mask);
    if (std::memcmp(h.magic, want.magic, sizeof(h.magic)) != 0 || h.version != want.version ||
        h.flowdev_bytes != want.flowdev_bytes)
        return fail(m, TUFRG_EINVAL, "not a checkpoint of this library version");
    if (h.precision != want.precision || h.ns != want.ns || h.nff != want.nff || h.Lq != want.Lq || h.nc != want.nc ||
        h.M != want.M || h.n_elems != want.n_elems || h.channel_mask != want.channel_mask || h.basis != want.basis ||
        h.regulator != want.regulator || h.loops_tc != want.loops_tc)
        return fail(m, TUFRG_EINVAL, "the checkpoint belongs to another model or channel mask");
    const size_t n = state_elems(m);
    const unsigned char *p = static_cast<const unsigned char *>(h_buf);
    // a state or derivative that is not finite would only surface as a failed step later, or not at all where it
    // sits outside the rows the symmetric path reads: refuse it here
    for (size_t i = 0; i < 4 * n; i++) {
        double v;
        std::memcpy(&v, p + sizeof(h) + sizeof(FlowDev) + i * sizeof(double), sizeof(v));
        if (!std::isfinite(v)) return fail(m, TUFRG_ENONFINITE, "the checkpoint holds a non-finite state or derivative");
    }
    // the launch shapes the checkpointed run used (they fix the summation order), then a fresh capture if needed
    // (both checked before either is changed, so that a refused checkpoint leaves the model as it was)
    if (h.products != m->products &&
        (m->precision == TUFRG_FP64 || (h.products != TUFRG_PRODUCTS_TC && h.products != TUFRG_PRODUCTS_SIMT)))
        return fail(m, TUFRG_EINVAL, "the checkpoint's products backend does not apply to this model");
    if (h.ky_chunks != m->plan.ky_chunks && (h.ky_chunks < 1 || h.ky_chunks > (int)m->plan_cand.size()))
        return fail(m, TUFRG_EINVAL, "the checkpoint's loop launch shape does not apply to this model");
    bool reshaped = false;
    if (h.products != m->products) {
        m->products = h.products;
        reshaped = true;
    }
    if (h.ky_chunks != m->plan.ky_chunks) {
        m->plan = m->plan_cand[h.ky_chunks - 1];
        reshaped = true;
    }
    if (reshaped && m->step_graph) {
        cudaGraphExecDestroy(m->step_graph);
        m->step_graph = nullptr;
    }
    if (reshaped) drop_rhs_graphs(m);
    cudaStream_t user;
    if ((st = flow_enter(m, &user)) != TUFRG_OK) return st;
    auto run = [&]() -> tufrg_status {
        tufrg_status s2 = flow_alloc(m);
        if (s2 != TUFRG_OK) return s2;
        std::memcpy(m->h_flow, p + sizeof(h), sizeof(FlowDev));
        CK(cudaMemcpyAsync(m->d_flow, m->h_flow, sizeof(FlowDev), cudaMemcpyHostToDevice, m->stream), "copy controller");
        CK(cudaMemcpyAsync(m->d_y, p + sizeof(h) + sizeof(FlowDev), sizeof(double2) * n, cudaMemcpyHostToDevice, m->stream),
           "copy state");
        // the projections of the restored state (the final report locates max |A| in them); the derivative goes to
        // a stage buffer that the next attempt overwrites, k1 itself comes from the checkpoint
        CK(launch_stage_scalars(m, m->d_flow, 0.0), "stage temperature");
        s2 = rhs_device(m, m->d_y, o->channel_mask, m->d_k[1], nullptr, true);
        if (s2 != TUFRG_OK) return s2;
        CK(cudaMemcpyAsync(m->d_k[0], p + sizeof(h) + sizeof(FlowDev) + sizeof(double2) * n, sizeof(double2) * n,
                           cudaMemcpyHostToDevice, m->stream), "copy derivative");
        if ((s2 = flow_capture(m, o->channel_mask)) != TUFRG_OK) return s2;
        CK(cudaStreamSynchronize(m->stream), "sync");
        return TUFRG_OK;
    };
    st = run();
    if (st != TUFRG_OK) {
        flow_leave(m, user);
        return st;
    }
    m->flow_open = true;
    m->flow_user = user;
    m->flow_mask = o->channel_mask;
    m->flow_t0 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
    return TUFRG_OK;
}

tufrg_status tufrg_flow_batch(tufrg_model *const *models, int n, const tufrg_flow_opts *o, tufrg_flow_result *res)
try {
    if (!models || n < 1 || !o || !res) return TUFRG_EINVAL;
    for (int i = 0; i < n; i++) {
        if (!models[i]) return TUFRG_EINVAL;
        for (int j = 0; j < i; j++)
            if (models[j] == models[i]) return fail(models[i], TUFRG_EINVAL, "a model appears twice in the batch");
        tufrg_status st = flow_check_args(models[i], o, &res[i]);
        if (st != TUFRG_OK) return st;
        if (models[i]->flow_open) return fail(models[i], TUFRG_EINVAL, "a stepwise flow is open on this model");
    }
    const auto t_start = std::chrono::steady_clock::now();
    std::vector<char> active(n, 1);
    std::vector<cudaStream_t> user(n, nullptr);
    std::vector<char> entered(n, 0);
    tufrg_status first = TUFRG_OK;
    for (int i = 0; i < n; i++) {
        std::memset(&res[i], 0, sizeof(res[i]));
        tufrg_status st = flow_enter(models[i], &user[i]);
        if (st == TUFRG_OK) {
            entered[i] = 1;
            st = flow_prepare(models[i], o);
        }
        if (st == TUFRG_OK && models[i]->h_flow->status != 0) {   // stopped before the first attempt
            active[i] = 0;
            st = read_device_error(models[i]);
            if (st == TUFRG_OK) st = flow_finish(models[i], nullptr, &res[i]);
        }
        if (st != TUFRG_OK) {
            active[i] = 0;
            if (first == TUFRG_OK) first = st;
        }
    }
    // lock-step rounds: every running flow replays one attempt on its own stream, then all are polled
    int running = 0;
    for (int i = 0; i < n; i++) running += active[i];
    while (running > 0) {
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            tufrg_model *m = models[i];
            cudaError_t e = cudaGraphLaunch(m->step_graph, m->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(m->h_flow, m->d_flow, sizeof(FlowDev), cudaMemcpyDeviceToHost, m->stream);
            if (e != cudaSuccess) {
                active[i] = 0;
                running--;
                if (first == TUFRG_OK) first = cuda_fail(m, e, "batched graph launch");
            }
        }
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            tufrg_model *m = models[i];
            cudaError_t e = cudaStreamSynchronize(m->stream);
            if (e != cudaSuccess || m->h_flow->status != 0) {
                active[i] = 0;
                running--;
                tufrg_status st = e != cudaSuccess ? cuda_fail(m, e, "sync") : read_device_error(m);
                if (st == TUFRG_OK) st = flow_finish(m, nullptr, &res[i]);
                if (st != TUFRG_OK && first == TUFRG_OK) first = st;
            }
        }
    }
    for (int i = 0; i < n; i++) {
        if (!entered[i]) continue;
        tufrg_status st = flow_leave(models[i], user[i]);
        if (st != TUFRG_OK && first == TUFRG_OK) first = st;
    }
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    for (int i = 0; i < n; i++) res[i].wall_s = wall;
    return first;
} catch (const std::exception &ex) {
    return host_alloc_fail(nullptr, ex);
}

}  // extern "C"

namespace tufrg {

// NVTX ranges named after the phases (host-side markers for profilers; no cost without an attached tool)
static const char *const kPhaseNames[PH_N] = {"tufrg fermi", "tufrg loops", "tufrg loop_reduce", "tufrg dft",
                                              "tufrg project", "tufrg vlv", "tufrg rk", "tufrg sym_scatter"};

PhaseScope::PhaseScope(tufrg_model *mm, int phase, int n_launch) : m(mm)
{
    nvtxRangePushA(kPhaseNames[phase]);
    m->launches += n_launch;
    if (phase == PH_LOOPS) m->loop_launches += n_launch;
    if (!m->timing) return;
    while (m->evpool.size() < m->evused + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        m->evpool.push_back(e);
    }
    tufrg_model::TimerRec r{phase, m->evpool[m->evused], m->evpool[m->evused + 1]};
    m->evused += 2;
    cudaEventRecord(r.a, m->stream);
    idx = (int)m->trec.size();
    m->trec.push_back(r);
}

PhaseScope::~PhaseScope()
{
    if (idx >= 0) cudaEventRecord(m->trec[idx].b, m->stream);
    nvtxRangePop();
}

}  // namespace tufrg

extern "C" {

tufrg_status tufrg_set_device_error(tufrg_model *m, int value)
{
    if (!m) return TUFRG_EINVAL;
    const int v = value ? 1 : 0;
    CK(cudaMemcpyAsync(m->d_err, &v, sizeof(int), cudaMemcpyHostToDevice, m->stream), "write error flag");
    CK(cudaStreamSynchronize(m->stream), "sync");
    return TUFRG_OK;
}

tufrg_status tufrg_timing_begin(tufrg_model *m)
{
    if (!m) return TUFRG_EINVAL;
    m->trec.clear();
    m->evused = 0;
    m->launches = 0;
    m->loop_launches = 0;
    m->timing = true;
    return TUFRG_OK;
}

tufrg_status tufrg_timing_end(tufrg_model *m, double *h_ms, int n_ms, long long *h_launches, long long *h_loop_launches)
{
    if (!m) return TUFRG_EINVAL;
    m->timing = false;
    CK(cudaStreamSynchronize(m->stream), "sync");
    double acc[PH_N] = {0};
    for (auto &r : m->trec) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b), "event time");
        acc[r.phase] += ms;
    }
    for (int i = 0; i < n_ms && i < PH_N; i++) h_ms[i] = acc[i];
    if (h_launches) *h_launches = m->launches;
    if (h_loop_launches) *h_loop_launches = m->loop_launches;
    m->trec.clear();
    m->evused = 0;
    return TUFRG_OK;
}

}  // extern "C"
