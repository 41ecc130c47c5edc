// plan.cu — host-side level plans (see plan.h).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include "launch.h"
#include "plan.h"
#include "sym.cuh"
#include "sttsm.h"

namespace sttsm {

int make_shape(int m, int64_t n, int64_t p, int b, Shape* s)
{
    if (m < 1 || n < 1 || p < 1 || b < 1) return STTSM_ERR_ARG;
    if (m > STTSM_MAX_M) return STTSM_ERR_UNSUPPORTED;
    s->m = m; s->b = b; s->n = n; s->p = p;
    s->nbar = (n + b - 1) / b;
    s->pbar = (p + b - 1) / b;
    double bmd = 1.0;
    for (int a = 0; a < m; ++a) bmd *= b;
    if (bmd >= 2147483647.0) return STTSM_ERR_UNSUPPORTED;   // b^m (in-block offsets) must fit int32
    s->bm = 1;
    for (int a = 0; a < m; ++a) s->bm *= b;
    s->R = s->bm / b;
    // every block count below must stay below 2^27 (ranks are packed with q)
    auto safe_binom = [](int64_t x, int y) -> int64_t {
        double c = 1.0;
        for (int i = 1; i <= y; ++i) c = c * (double)(x - y + i) / i;
        if (x < y) return 0;
        if (c >= 134217728.0) return -1;
        return binom_small(x, y);
    };
    s->buf_elems[0] = s->buf_elems[1] = 0;
    for (int d = 0; d < m; ++d) {
        LevelShape& L = s->lv[d];
        L.d = d;
        L.k = m - 1 - d;
        L.nodes_parent = d == 0 ? 1 : safe_binom(s->pbar + d - 1, d);
        L.nodes_out = safe_binom(s->pbar + d, d + 1);
        L.P_parent = safe_binom(s->nbar + L.k, L.k + 1);
        L.P_out = L.k == 0 ? 1 : safe_binom(s->nbar + L.k - 1, L.k);
        if (L.nodes_parent < 0 || L.nodes_out < 0 || L.P_parent < 0 || L.P_out < 0) return STTSM_ERR_UNSUPPORTED;
        if ((double)L.P_out * (double)s->R >= 2147483647.0) return STTSM_ERR_UNSUPPORTED;
        if (d < m - 1) {
            int64_t e = L.nodes_out * L.P_out * s->bm;
            if (e > s->buf_elems[d & 1]) s->buf_elems[d & 1] = e;
        }
    }
    return STTSM_OK;
}

void build_level_G(const Shape& s, int d, std::vector<int32_t>& G)
{
    const LevelShape& L = s.lv[d];
    const int k = L.k;
    G.resize((size_t)(L.P_out * s.nbar));
    int32_t prefix[STTSM_MAX_M], stored[STTSM_MAX_M];
    for (int64_t pr = 0; pr < L.P_out; ++pr) {
        if (k > 0) colex_unrank(pr, k, prefix);
        for (int64_t ib = 0; ib < s.nbar; ++ib) {
            // insert ib before the first prefix entry >= ib; q = its position
            int q = 0;
            while (q < k && prefix[q] < ib) ++q;
            for (int t = 0; t < q; ++t) stored[t] = prefix[t];
            stored[q] = (int32_t)ib;
            for (int t = q; t < k; ++t) stored[t + 1] = prefix[t];
            const int64_t rank = colex_rank(stored, k + 1);
            G[(size_t)(pr * s.nbar + ib)] = (int32_t)((rank << 3) | q);
        }
    }
    // offset table OFF[q][rr] = rr % b^q + b^(q+1) (rr / b^q), q = 0..k, appended after G
    const size_t base = G.size();
    G.resize(base + (size_t)(k + 1) * s.R);
    int64_t bq = 1;
    for (int q = 0; q <= k; ++q, bq *= s.b)
        for (int64_t rr = 0; rr < s.R; ++rr)
            G[base + (size_t)(q * s.R + rr)] = (int32_t)(rr % bq + bq * s.b * (rr / bq));
}

bool tma_order16x8(const Shape& s, int d)
{
    if (!tc_tma_mode(s) || !tma_sw32(s) || s.m > 4 || s.m < 3 || s.b % 16 != 0 || (s.R / s.b) % 8 != 0) return false;
    const int k = s.lv[d].k;
    int64_t bq = s.b;
    for (int q = 1; q <= k; ++q, bq *= s.b)
        if (bq % 128 != 0 && 128 % bq != 0) return true;
    return false;
}

void build_level_tiles(const Shape& s, int d, int BM, int BN, int32_t inst, std::vector<Tile>& tiles, bool order16x8)
{
    const LevelShape& L = s.lv[d];
    const int64_t rows = L.P_out * s.R;
    // first rows of the tiles of one parent: row0 + t, or blocks of 16 fastest x 8 next
    std::vector<int64_t> starts;
    if (order16x8) {
        for (int64_t pr = 0; pr < L.P_out; ++pr)
            for (int64_t s0 = 0; s0 < s.R / s.b; s0 += 8)
                for (int64_t f0 = 0; f0 < s.b; f0 += 16) starts.push_back(pr * s.R + f0 + s.b * s0);
    } else {
        for (int64_t r0 = 0; r0 < rows; r0 += BM) starts.push_back(r0);
    }
    int32_t u[STTSM_MAX_M];
    for (int64_t par = 0; par < L.nodes_parent; ++par) {
        int64_t children, child_base = 0;
        if (d == 0) {
            children = s.pbar;
        } else {
            colex_unrank(par, d, u);   // parent (jbar_{k+1} <= ... <= jbar_{m-1})
            children = (int64_t)u[0] + 1;
            for (int t = 0; t < d; ++t) child_base += binom_small((int64_t)u[t] + t + 1, t + 2);
        }
        const int64_t ncols = children * s.b;
        // wide tiles (BN >= 128): a parent's columns are cut into equal widths (a
        // multiple of 16) rather than full tiles plus a narrow remainder
        int64_t w = BN;
        const int64_t nct = (ncols + BN - 1) / BN;
        if (BN >= 128 && nct > 1) w = ((ncols + nct - 1) / nct + 15) / 16 * 16;
        for (int64_t r0 : starts) {
            for (int64_t c0 = 0; c0 < ncols; c0 += w) {
                Tile t;
                t.inst = inst;
                t.parent = (int32_t)par;
                t.child_base = (int32_t)child_base;
                t.row0 = (int32_t)r0;
                t.col0 = (int32_t)c0;
                t.ncols = (int32_t)(ncols - c0 < w ? ncols - c0 : w);
                t.pad0 = order16x8 ? 1 : 0;
                t.pad1 = 0;
                tiles.push_back(t);
            }
        }
    }
}

// m <= 5: a row then has at most 4! = 24 mirrors, the length of the store's list.
bool sym_shape_ok(const Shape& s) { return s.m <= 5 && s.nbar * s.b <= 64 && s.b <= 64 && s.pbar < 65536; }

void build_level_tiles_sym(const Shape& s, int d, int BM, int BN, int32_t inst, std::vector<Tile>& tiles)
{
    const LevelShape& L = s.lv[d];
    SymTab T;
    sym_tab_fill(T, 0, 1);
    const int Kp = (int)(s.nbar * s.b);
    int32_t u[STTSM_MAX_M];
    for (int64_t par = 0; par < L.nodes_parent; ++par) {
        int64_t children, child_base = 0;
        uint32_t pattern = 0;
        int u0 = 0;
        if (d == 0) {
            children = s.pbar;
        } else {
            colex_unrank(par, d, u);   // parent (jbar_{k+1} <= ... <= jbar_{m-1})
            children = (int64_t)u[0] + 1;
            u0 = u[0];
            for (int t = 0; t < d; ++t) child_base += binom_small((int64_t)u[t] + t + 1, t + 2);
            for (int t = 0; t + 1 < d; ++t)
                if (u[t] == u[t + 1]) pattern |= 1u << t;
        }
        const int64_t rows = sym_parent_rows(T, s.m, L.k, s.b, Kp, pattern);
        const int64_t ncols = children * s.b;
        for (int64_t r0 = 0; r0 < rows; r0 += BM) {
            for (int64_t c0 = 0; c0 < ncols; c0 += BN) {
                Tile t;
                t.inst = inst;
                t.parent = (int32_t)par;
                t.child_base = (int32_t)child_base;
                t.row0 = (int32_t)r0;
                t.col0 = (int32_t)c0;
                t.ncols = (int32_t)(ncols - c0 < BN ? ncols - c0 : BN);
                t.pad0 = SYM_TILE | (int32_t)(pattern << 8) | (int32_t)((uint32_t)u0 << 16);
                t.pad1 = (int32_t)rows;
                tiles.push_back(t);
            }
        }
    }
}

int64_t level_tile_count(const Shape& s, int d, int BM, int BN)
{
    const LevelShape& L = s.lv[d];
    const int64_t row_tiles = (L.P_out * s.R + BM - 1) / BM;
    int32_t u[STTSM_MAX_M];
    int64_t count = 0;
    for (int64_t par = 0; par < L.nodes_parent; ++par) {
        int64_t children = s.pbar;
        if (d > 0) {
            colex_unrank(par, d, u);
            children = (int64_t)u[0] + 1;
        }
        const int64_t ncols = children * s.b;
        int64_t w = BN;
        const int64_t nct = (ncols + BN - 1) / BN;
        if (BN >= 128 && nct > 1) w = ((ncols + nct - 1) / nct + 15) / 16 * 16;
        count += row_tiles * ((ncols + w - 1) / w);
    }
    return count;
}

int pair_group(const Shape& s)
{
    const int64_t Kc = (s.nbar * s.b + 3) & ~(int64_t)3;
    const int64_t S_total = s.R / s.b;
    const int64_t g = PAIR_ROWS / Kc;
    return (int)(g < S_total ? g : S_total);
}

bool pair_mode(const Shape& s)
{
    if (s.m < 2 || s.nbar * s.b > 64 || s.pbar * s.b > 64) return false;
    const int64_t Kc = (s.nbar * s.b + 3) & ~(int64_t)3;
    const int64_t Gs = pair_group(s);
    if (Gs < 1) return false;
    const int64_t RBp = (s.b * Gs + 3) & ~(int64_t)3;
    return Kc * s.pbar * RBp <= PAIR_U_MAX;
}

void build_pair_tiles(const Shape& s, int32_t inst, std::vector<Tile>& tiles)
{
    const int d = s.m - 2;
    const LevelShape& L = s.lv[d];
    const int Gs = pair_group(s);
    const int64_t S_total = s.R / s.b;
    int32_t u[STTSM_MAX_M];
    for (int64_t par = 0; par < L.nodes_parent; ++par) {
        int64_t children = s.pbar, cbase = 0;
        if (d > 0) {
            colex_unrank(par, d, u);   // J = (jbar_2 <= ... <= jbar_{m-1})
            children = (int64_t)u[0] + 1;
            for (int t = 0; t < d; ++t) cbase += binom_small((int64_t)u[t] + t + 2, t + 3);
        }
        for (int64_t s0 = 0; s0 < S_total; s0 += Gs) {
            Tile t;
            t.inst = inst;
            t.parent = (int32_t)par;
            t.child_base = 0;
            t.row0 = (int32_t)s0;
            t.col0 = (int32_t)children;
            t.ncols = Gs;
            t.pad0 = (int32_t)cbase;
            t.pad1 = 0;
            tiles.push_back(t);
        }
    }
}

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int64_t, int64_t, int, int, int, int, bool>, DevPlan*> g_plans;

void free_plan(DevPlan* P)
{
    for (int d = 0; d < STTSM_MAX_M; ++d) {
        if (P->d_tiles[d]) cudaFree(P->d_tiles[d]);
        if (P->d_G[d]) cudaFree(P->d_G[d]);
    }
    if (P->d_pair) cudaFree(P->d_pair);
    delete P;
}
}  // namespace

const DevPlan* get_dev_plan(int m, int64_t n, int64_t p, int b, int BM, int BN, int bn_last, bool sym)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (bn_last <= 0) bn_last = BN;
    auto key = std::make_tuple(dev, m, n, p, b, BM, BN, bn_last, sym);
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) return it->second;
    DevPlan* P = new DevPlan();
    for (int d = 0; d < STTSM_MAX_M; ++d) { P->d_tiles[d] = nullptr; P->d_G[d] = nullptr; P->ntiles[d] = 0; P->maxcols[d] = 0; }
    P->d_pair = nullptr;
    P->npair = 0;
    if (make_shape(m, n, p, b, &P->shape) != STTSM_OK) { delete P; return nullptr; }
    P->BM = BM;
    P->BN = BN;
    for (int d = 0; d < m; ++d) {
        std::vector<Tile> tiles;
        std::vector<int32_t> G;
        if (sym)
            build_level_tiles_sym(P->shape, d, BM, d == m - 1 ? bn_last : BN, 0, tiles);
        else
            build_level_tiles(P->shape, d, BM, d == m - 1 ? bn_last : BN, 0, tiles,
                              BM == TC_BM && tma_order16x8(P->shape, d));
        build_level_G(P->shape, d, G);
        P->ntiles[d] = (int)tiles.size();
        for (const Tile& t : tiles) P->maxcols[d] = std::max(P->maxcols[d], (int)t.ncols);
        if (cudaMalloc(&P->d_tiles[d], tiles.size() * sizeof(Tile)) != cudaSuccess ||
            cudaMalloc(&P->d_G[d], G.size() * sizeof(int32_t)) != cudaSuccess ||
            cudaMemcpy(P->d_tiles[d], tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(P->d_G[d], G.data(), G.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
            free_plan(P);
            return nullptr;
        }
    }
    if (BM == TC_BM && pair_mode(P->shape)) {
        std::vector<Tile> tiles;
        build_pair_tiles(P->shape, 0, tiles);
        P->npair = (int)tiles.size();
        if (cudaMalloc(&P->d_pair, tiles.size() * sizeof(Tile)) != cudaSuccess ||
            cudaMemcpy(P->d_pair, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice) != cudaSuccess) {
            free_plan(P);
            return nullptr;
        }
    }
    g_plans[key] = P;
    return P;
}

}  // namespace sttsm
