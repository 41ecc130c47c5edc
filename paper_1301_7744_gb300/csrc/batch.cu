// batch.cu — many independent sttsm instances per launch (sttsm_batch_*),
// and the block-size autotuner (sttsm_autotune_b).
//
// A batch plan groups the instances into waves whose workspaces fit the
// caller's budget.  Per wave: one launch splits every instance's X (split
// precisions), then one launch per level d runs the level-d tiles of every
// instance with m > d — the level kernels take a per-instance descriptor
// table, so instances of different m, n, p and b share each launch.  The
// whole sequence is captured once into a CUDA graph and replayed.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>
#include "launch.h"
#include "plan.h"
#include "sttsm.h"

using namespace sttsm;

namespace {

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

int npiece(int prec) { return prec_npiece(prec); }

// Cost model of one level launch's tiles, in SM cycles: each stage of a tile
// costs the larger of its MMA time (products x 2 K-steps x N/2 cycles for a
// 128 x N x 16 MMA) and the stage's operand-supply floor, and each tile adds a
// fixed cost (set-up, flushes, stores).  The floors and tile costs differ by
// kernel: TMA-fed (operands by TMA, no gather), gathered (per-stage gather
// latency), small-tile (two CTAs per SM, latency-bound tiles).
struct KernelCost { double stage_floor, tile; };

KernelCost kernel_cost(const Shape& s)
{
    if (tc_small_mode(s)) return {700.0, 4000.0};
    if (tc_tma_mode(s)) return {300.0, 3000.0};
    return {1100.0, 3000.0};
}

double tile_cost(int nk, int ncols, int nprod, const KernelCost& k)
{
    const double n16 = (double)((ncols + 15) & ~15);
    const double mma = nprod * 2.0 * n16 / 2.0;
    return nk * std::max(mma, k.stage_floor) + k.tile;
}

double plan_cost(const Shape& s, int prec, int BM, int BN)
{
    const int nprod = prec_npiece(prec) == 2 ? 3 : 6;
    if (tc_small_mode(s)) BN = TC_SMALL_BN;
    const KernelCost k = kernel_cost(s);
    double c = 0.0;
    for (int d = 0; d < s.m; ++d) {
        std::vector<Tile> tiles;
        build_level_tiles(s, d, BM, BN, 0, tiles);
        const int nk = (int)((s.nbar * s.b + TC_KC - 1) / TC_KC);
        for (const Tile& t : tiles) c += tile_cost(nk, t.ncols, nprod, k);
    }
    return c;
}

struct Instance {
    sttsm_desc desc;
    Shape shape;
    bool fused = false;         // last two levels in the fused launch
    bool sym = false;           // canonical entries only (in-block symmetry, sym.cuh)
    size_t ws_bytes;
    size_t x_off, buf_off[2];   // offsets inside the instance's workspace slice
    int rows, Kp;
    double cost;
};

struct LevelLaunch {
    int ntiles = 0;
    int maxcols = 0;              // widest tile
    int sym = 0;                  // some tiles in the in-block-symmetry mode
    Tile* d_tiles = nullptr;
    void* d_insts = nullptr;      // TcInst[] or LevelInst[]
    std::vector<int> inst_ids;    // instance of every descriptor
};

struct Wave {
    std::vector<int> ids;         // instances in this wave
    std::vector<size_t> ws_off;   // each instance's slice offset in the workspace
    int max_m = 0;
    SplitDesc* d_split = nullptr;
    int split_blocks = 0;
    LevelLaunch lv[STTSM_MAX_M][2];   // [level][0: regular tiles, 1: small-tile kernel]
    LevelLaunch pair;                  // fused last two levels of the short contractions, after every level
};

}  // namespace

struct sttsm_batch_plan_s {
    int prec = 0;
    std::vector<Instance> inst;
    std::vector<Wave> waves;
    std::map<std::tuple<int, int64_t, int, int>, int32_t*> G;   // (m, nbar, b, level) -> device G + OFF tables
    size_t ws_bytes = 0;
    // graph of the last run
    void* graph_ws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    int* status = nullptr;
    double useful_flops = 0.0;
};

namespace {

void destroy_plan(sttsm_batch_plan_s* P)
{
    if (!P) return;
    for (Wave& w : P->waves) {
        if (w.d_split) cudaFree(w.d_split);
        for (int d = 0; d < STTSM_MAX_M; ++d)
            for (int k = 0; k < 2; ++k) {
                if (w.lv[d][k].d_tiles) cudaFree(w.lv[d][k].d_tiles);
                if (w.lv[d][k].d_insts) cudaFree(w.lv[d][k].d_insts);
            }
        if (w.pair.d_tiles) cudaFree(w.pair.d_tiles);
        if (w.pair.d_insts) cudaFree(w.pair.d_insts);
    }
    for (auto& kv : P->G) cudaFree(kv.second);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->capture_stream) cudaStreamDestroy(P->capture_stream);
    delete P;
}

// Fills every level descriptor of every wave for the workspace `ws` (the
// descriptors hold absolute pointers, so they change with the workspace).
int bind_workspace(sttsm_batch_plan_s* P, char* ws)
{
    const bool fp64 = P->prec == STTSM_FP64;
    const int np = npiece(P->prec);
    for (Wave& w : P->waves) {
        std::vector<SplitDesc> sd;
        int64_t blocks = 0;
        std::vector<CUtensorMap> maps(w.ids.size());
        for (size_t a = 0; a < w.ids.size(); ++a) {
            const Instance& I = P->inst[w.ids[a]];
            char* base = ws + w.ws_off[a];
            if (!fp64) {
                SplitDesc s;
                s.X = (const float*)I.desc.X;
                s.out = base + I.x_off;
                s.p = (int)I.desc.p; s.n = (int)I.desc.n; s.rows = I.rows; s.Kp = I.Kp;
                s.first_block = blocks;
                blocks += ((int64_t)I.rows * I.Kp + 255) / 256;
                sd.push_back(s);
                const int box = tc_small_mode(I.shape) ? TC_SMALL_BN : TC_BN;
                if (make_x_tensor_map(&maps[a], base + I.x_off, np, I.rows, I.Kp, box) != STTSM_OK) return STTSM_ERR_CUDA;
            }
        }
        if (!fp64) {
            w.split_blocks = (int)blocks;
            if (!w.d_split && cudaMalloc(&w.d_split, sd.size() * sizeof(SplitDesc)) != cudaSuccess) return STTSM_ERR_NOMEM;
            if (cudaMemcpy(w.d_split, sd.data(), sd.size() * sizeof(SplitDesc), cudaMemcpyHostToDevice) != cudaSuccess)
                return STTSM_ERR_CUDA;
        }
        // position of every instance in the wave
        std::map<int, size_t> pos;
        for (size_t a = 0; a < w.ids.size(); ++a) pos[w.ids[a]] = a;
        for (int d = 0; d <= w.max_m; ++d)
        for (int mode = 0; mode < 2; ++mode) {
            // d == w.max_m: the pair launch (each instance at its own level m - 2)
            const bool pairl = d == w.max_m;
            if (pairl && mode == 1) continue;
            LevelLaunch& L = pairl ? w.pair : w.lv[d][mode];
            if (L.inst_ids.empty()) continue;
            std::vector<TcInst> tci(L.inst_ids.size());
            std::vector<LevelInst> lvi(L.inst_ids.size());
            for (size_t e = 0; e < L.inst_ids.size(); ++e) {
                const int id = L.inst_ids[e];
                const Instance& I = P->inst[id];
                const Shape& s = I.shape;
                const int dl = pairl ? s.m - 2 : d;
                const LevelShape& LS = s.lv[dl];
                char* base = ws + w.ws_off[pos[id]];
                LevelInst li;
                memset(&li, 0, sizeof(li));
                li.parent = dl == 0 ? I.desc.A : (const void*)(base + I.buf_off[(dl - 1) & 1]);
                li.out = (dl == s.m - 1 || pairl) ? I.desc.C : (void*)(base + I.buf_off[dl & 1]);
                li.sym_full = dl == s.m - 1 ? 1 : 0;
                li.G = P->G.at(std::make_tuple(s.m, s.nbar, s.b, dl));
                li.OFF = li.G + level_G_size(s, dl);
                li.X = I.desc.X;
                li.m = s.m; li.b = s.b; li.k = LS.k; li.nbar = (int32_t)s.nbar;
                li.n = (int32_t)s.n; li.p = (int32_t)s.p;
                li.R = (int32_t)s.R;
                li.Ktot = (int32_t)(s.nbar * s.b);
                li.bm = s.bm;
                li.P_parent = LS.P_parent;
                li.P_out = LS.P_out;
                li.rows_per_parent = LS.P_out * s.R;
                int64_t bp = 1;
                for (int q = 0; q <= STTSM_MAX_M; ++q) { li.bpow[q] = (int32_t)(bp < ((int64_t)1 << 31) ? bp : 0); bp *= s.b; }
                lvi[e] = li;
                memset(&tci[e], 0, sizeof(TcInst));
                if (!fp64) tci[e].tmX = maps[pos[id]];
                tci[e].L = li;
            }
            const size_t bytes = fp64 ? lvi.size() * sizeof(LevelInst) : tci.size() * sizeof(TcInst);
            if (!L.d_insts && cudaMalloc(&L.d_insts, bytes) != cudaSuccess) return STTSM_ERR_NOMEM;
            const void* src = fp64 ? (const void*)lvi.data() : (const void*)tci.data();
            if (cudaMemcpy(L.d_insts, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return STTSM_ERR_CUDA;
        }
    }
    return STTSM_OK;
}

int enqueue(sttsm_batch_plan_s* P, cudaStream_t s)
{
    const bool fp64 = P->prec == STTSM_FP64;
    const bool r64 = prec_r64(P->prec);
    const int np = npiece(P->prec);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    for (Wave& w : P->waves) {
        if (!fp64 && w.split_blocks > 0) {
            if (launch_split_x_batch(w.d_split, (int)w.ids.size(), w.split_blocks, np, s) != 0) return STTSM_ERR_CUDA;
        }
        for (int d = 0; d < w.max_m; ++d)
        for (int mode = 0; mode < 2; ++mode) {
            LevelLaunch& L = w.lv[d][mode];
            if (L.ntiles == 0) continue;
            TcInst dummy;
            memset(&dummy, 0, sizeof(dummy));
            const TcInst* ti = (const TcInst*)L.d_insts;
            // under the R64 precisions every gathered launch sums in FP64 (its tiles are at
            // most 128 wide) and the FP32 kernel does so at each instance's last level
            const int rc = fp64 ? launch_level_fp64(dummy.L, (const LevelInst*)L.d_insts, L.d_tiles, L.ntiles, sms, s)
                         : (mode && (small_kernel_kind() == 0 || r64))
                             ? launch_level_small_f32_tc(ti, L.d_tiles, L.ntiles, sms, s, r64 ? 1 : 0, L.sym)
                         : mode ? launch_level_tc_small(np, dummy, ti, L.d_tiles, L.ntiles, sms, P->status, s)
                         : r64 ? launch_level_tc_r64(np, dummy, ti, L.d_tiles, L.ntiles, sms, P->status, L.maxcols, s)
                               : launch_level_tc(np, dummy, ti, L.d_tiles, L.ntiles, sms, P->status, s);
            if (rc != 0) return STTSM_ERR_CUDA;
        }
        if (w.pair.ntiles > 0 &&
            launch_level_pair_f32_tc((const TcInst*)w.pair.d_insts, w.pair.d_tiles, w.pair.ntiles, sms, s) != 0)
            return STTSM_ERR_CUDA;
    }
    return STTSM_OK;
}

}  // namespace

namespace sttsm {
int* batch_status_word();   // defined in capi.cu
}

extern "C" {

int sttsm_autotune_b(int m, int64_t n, int64_t p, int prec, const int* cands, int ncand)
{
    if (!cands || ncand <= 0) return STTSM_ERR_ARG;
    int best = -1;
    double best_cost = 0.0;
    for (int c = 0; c < ncand; ++c) {
        Shape s;
        if (cands[c] < 1 || make_shape(m, n, p, cands[c], &s) != STTSM_OK) continue;
        const double cost = prec == STTSM_FP64 ? (double)sttsm_flops(m, n, p, cands[c])
                                               : plan_cost(s, prec, TC_BM, TC_BN);
        if (best < 0 || cost < best_cost) { best = cands[c]; best_cost = cost; }
    }
    return best < 0 ? STTSM_ERR_UNSUPPORTED : best;
}

int sttsm_batch_plan_create(const sttsm_desc* d, int count, int prec, size_t ws_budget, void** plan_out)
{
    if (!d || count <= 0 || !plan_out) return STTSM_ERR_ARG;
    if (prec == STTSM_TF32X3) return STTSM_ERR_UNSUPPORTED;
    if (!prec_valid(prec)) return STTSM_ERR_ARG;
    const bool fp64 = prec == STTSM_FP64;
    const int np = npiece(prec);
    const size_t esz = fp64 ? 8 : 4;
    const int BM = fp64 ? 64 : TC_BM, BN = fp64 ? 64 : TC_BN;
    std::unique_ptr<sttsm_batch_plan_s, void (*)(sttsm_batch_plan_s*)> P(new sttsm_batch_plan_s(), destroy_plan);
    P->prec = prec;
    P->status = batch_status_word();
    if (!P->status) return STTSM_ERR_CUDA;
    P->inst.resize(count);
    for (int i = 0; i < count; ++i) {
        Instance& I = P->inst[i];
        I.desc = d[i];
        if (!d[i].A || !d[i].X || !d[i].C) return STTSM_ERR_ARG;
        if (((uintptr_t)d[i].A | (uintptr_t)d[i].X | (uintptr_t)d[i].C) % 16 != 0) return STTSM_ERR_ARG;
        if (d[i].n >= ((int64_t)1 << 30) || d[i].p >= ((int64_t)1 << 30)) return STTSM_ERR_UNSUPPORTED;
        int rc = make_shape(d[i].m, d[i].n, d[i].p, d[i].b, &I.shape);
        if (rc != STTSM_OK) return rc;
        const Shape& s = I.shape;
        I.rows = (int)(s.pbar * s.b);
        I.Kp = (int)(((s.nbar * s.b) + 7) / 8 * 8);
        size_t off = 0;
        I.x_off = 0;
        off = np ? up256((size_t)np * I.rows * I.Kp * 2) : 0;
        I.buf_off[0] = off;
        off += up256((size_t)s.buf_elems[0] * esz);
        I.buf_off[1] = off;
        off += up256((size_t)s.buf_elems[1] * esz);
        I.ws_bytes = std::max<size_t>(off, 256);
        I.sym = !fp64 && sym_levels(s, prec);
        I.fused = !fp64 && !prec_r64(prec) && tc_small_mode(s) && small_kernel_kind() == 0 && fused_tail_in_batches() &&
                  pair_mode(s) && !I.sym;
        I.cost = sttsm_flops(s.m, s.n, s.p, s.b);
        P->useful_flops += I.cost;
        if (ws_budget && I.ws_bytes > ws_budget) return STTSM_ERR_NOMEM;
    }
    // waves: heaviest instances first, greedily packed under the budget
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P->inst[a].cost > P->inst[b].cost; });
    size_t used = 0;
    for (int id : order) {
        const size_t need = P->inst[id].ws_bytes;
        if (P->waves.empty() || (ws_budget && used + need > ws_budget)) {
            P->waves.emplace_back();
            used = 0;
        }
        Wave& w = P->waves.back();
        w.ids.push_back(id);
        w.ws_off.push_back(used);
        used += need;
        P->ws_bytes = std::max(P->ws_bytes, used);
        w.max_m = std::max(w.max_m, P->inst[id].shape.m);
    }
    // G tables shared by (m, nbar, level); tile lists per wave and level
    for (const Instance& I : P->inst) {
        for (int lv = 0; lv < I.shape.m; ++lv) {
            auto key = std::make_tuple(I.shape.m, I.shape.nbar, I.shape.b, lv);
            if (P->G.count(key)) continue;
            std::vector<int32_t> G;
            build_level_G(I.shape, lv, G);
            int32_t* dG = nullptr;
            if (cudaMalloc(&dG, G.size() * sizeof(int32_t)) != cudaSuccess) return STTSM_ERR_NOMEM;
            P->G[key] = dG;
            if (cudaMemcpy(dG, G.data(), G.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
                return STTSM_ERR_CUDA;
        }
    }
    for (Wave& w : P->waves) {
        for (int lv = 0; lv < w.max_m; ++lv)
        for (int mode = 0; mode < 2; ++mode) {
            LevelLaunch& L = w.lv[lv][mode];
            std::vector<Tile> tiles;
            for (int id : w.ids) {
                const Instance& I = P->inst[id];
                if (I.shape.m <= lv) continue;
                const bool small = !fp64 && tc_small_mode(I.shape);
                if ((int)small != mode) continue;
                if (I.fused && lv >= I.shape.m - 2) continue;   // in the pair launch
                const int32_t e = (int32_t)L.inst_ids.size();
                L.inst_ids.push_back(id);
                if (small && I.sym) {
                    build_level_tiles_sym(I.shape, lv, BM, TC_SMALL_BN, e, tiles);
                    L.sym = 1;
                } else {
                    build_level_tiles(I.shape, lv, BM, small ? TC_SMALL_BN : (prec_r64(prec) ? R64_BN : BN), e, tiles);
                }
            }
            L.ntiles = (int)tiles.size();
            for (const Tile& t : tiles) L.maxcols = std::max(L.maxcols, (int)t.ncols);
            if (L.ntiles == 0) continue;
            if (cudaMalloc(&L.d_tiles, tiles.size() * sizeof(Tile)) != cudaSuccess) return STTSM_ERR_NOMEM;
            if (cudaMemcpy(L.d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice) != cudaSuccess)
                return STTSM_ERR_CUDA;
        }
        LevelLaunch& L = w.pair;
        std::vector<Tile> tiles;
        for (int id : w.ids) {
            const Instance& I = P->inst[id];
            if (!I.fused) continue;
            const int32_t e = (int32_t)L.inst_ids.size();
            L.inst_ids.push_back(id);
            build_pair_tiles(I.shape, e, tiles);
        }
        L.ntiles = (int)tiles.size();
        if (L.ntiles > 0) {
            if (cudaMalloc(&L.d_tiles, tiles.size() * sizeof(Tile)) != cudaSuccess) return STTSM_ERR_NOMEM;
            if (cudaMemcpy(L.d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice) != cudaSuccess)
                return STTSM_ERR_CUDA;
        }
    }
    *plan_out = P.release();
    return STTSM_OK;
}

int sttsm_batch_workspace_size(const void* plan, size_t* bytes)
{
    if (!plan || !bytes) return STTSM_ERR_ARG;
    *bytes = ((const sttsm_batch_plan_s*)plan)->ws_bytes;
    return STTSM_OK;
}

int sttsm_batch_info(const void* plan, int* waves, double* useful_flops)
{
    if (!plan) return STTSM_ERR_ARG;
    const sttsm_batch_plan_s* P = (const sttsm_batch_plan_s*)plan;
    if (waves) *waves = (int)P->waves.size();
    if (useful_flops) *useful_flops = P->useful_flops;
    return STTSM_OK;
}

int sttsm_batch_run(void* plan, void* workspace, size_t ws_bytes, void* stream)
{
    sttsm_batch_plan_s* P = (sttsm_batch_plan_s*)plan;
    if (!P) return STTSM_ERR_ARG;
    if (ws_bytes < P->ws_bytes || (P->ws_bytes && (!workspace || (uintptr_t)workspace % 256))) return STTSM_ERR_NOMEM;
    if (!P->exec || P->graph_ws != workspace) {
        if (P->exec) { cudaGraphExecDestroy(P->exec); P->exec = nullptr; }
        if (P->graph) { cudaGraphDestroy(P->graph); P->graph = nullptr; }
        int rc = bind_workspace(P, (char*)workspace);
        if (rc != STTSM_OK) return rc;
        if (!P->capture_stream && cudaStreamCreateWithFlags(&P->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return STTSM_ERR_CUDA;
        if (cudaStreamBeginCapture(P->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return STTSM_ERR_CUDA;
        rc = enqueue(P, P->capture_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(P->capture_stream, &g);
        if (rc != STTSM_OK || e != cudaSuccess) { if (g) cudaGraphDestroy(g); return rc != STTSM_OK ? rc : STTSM_ERR_CUDA; }
        P->graph = g;
        if (cudaGraphInstantiate(&P->exec, g, 0) != cudaSuccess) return STTSM_ERR_CUDA;
        P->graph_ws = workspace;
    }
    return cudaGraphLaunch(P->exec, (cudaStream_t)stream) == cudaSuccess ? STTSM_OK : STTSM_ERR_CUDA;
}

int sttsm_batch_plan_destroy(void* plan)
{
    destroy_plan((sttsm_batch_plan_s*)plan);
    return STTSM_OK;
}

int sttsm_batch(const sttsm_desc* d, int count, int prec, void* workspace, size_t ws_bytes, void* stream)
{
    void* plan = nullptr;
    int rc = sttsm_batch_plan_create(d, count, prec, ws_bytes, &plan);
    if (rc != STTSM_OK) return rc;
    rc = sttsm_batch_run(plan, workspace, ws_bytes, stream);
    if (rc == STTSM_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = STTSM_ERR_CUDA;
    sttsm_batch_plan_destroy(plan);
    return rc;
}

}  // extern "C"
