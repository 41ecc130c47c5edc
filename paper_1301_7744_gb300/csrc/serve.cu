// serve.cu — continuous-batching serving of sttsm requests (sttsm_serve_*).
//
// A serve handle owns an HBM arena of the caller's budget (workspaces of
// admitted requests: X pieces and temporaries), one CUDA stream and a
// scheduler thread.  Requests wait in a FIFO queue until their workspace fits
// in the arena; admitted requests advance one level of the algorithm-by-
// blocks (Fig. 5) per step, and a step is one set of launches covering every
// active request at its own current level — requests that arrive while others
// run join at the next step and share its launches (continuous batching).
// A request's last level is tagged with the step's CUDA event; when the event
// completes the request is done, its latency (submit -> completion seen by the
// scheduler) is recorded and its workspace returns to the arena.  Up to two
// steps are in flight, so the host builds step s+1 while the GPU runs step s.
//
// Nothing in the scheduler loop allocates device or pinned memory or waits for
// the whole stream: the level tables (G) live in a table region reserved at
// create time (first-fit, entries of shapes no active request uses are evicted
// when it is full), the per-step staging buffers (pinned host + device) have a
// fixed size (a step takes active requests in turn until its staging is full;
// the others advance at the next step), and the step events come from a fixed
// pool.  Admission takes queued requests in arrival order but lets a later
// request pass one whose workspace does not fit yet, until the waiting one is
// older than SERVE_AGE_CAP_S: from then on nothing passes it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>
#include "launch.h"
#include "plan.h"
#include "sym.cuh"
#include "sttsm.h"

using namespace sttsm;

namespace sttsm {
int* batch_status_word();   // capi.cu
int peek_status_word();     // capi.cu
}

namespace {

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t SERVE_TABLE_BYTES = (size_t)64 << 20;     // level tables (G), outside the budget
constexpr size_t SERVE_STAGING_BYTES = (size_t)32 << 20;   // per staging buffer (two), outside the budget
constexpr double SERVE_AGE_CAP_S = 0.020;                  // later requests stop passing one older than this
constexpr int SERVE_EVENTS = 4;                            // step events (at most two steps in flight)
constexpr int SERVE_PASS_WINDOW = 64;                      // queued requests looked at per admission round
constexpr size_t SERVE_UPLOAD_BYTES = (size_t)4 << 20;     // pinned buffer for level-table uploads
constexpr size_t SERVE_STAGING_SLACK = 4096;               // alignment of a step's staging segments

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing of freed neighbours.
class Arena {
public:
    explicit Arena(size_t size) : size_(size) { free_[0] = size; }
    bool alloc(size_t n, size_t* off)
    {
        n = up256(n ? n : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = up256(n ? n : 1);
        used_ -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;
};

enum { Q_QUEUED = 0, Q_ACTIVE = 1, Q_FINISHING = 2, Q_DONE = 3 };

struct Req {
    sttsm_desc d;
    Shape s;
    bool small = false;
    bool tma = false;           // TMA-fed kernel: A split once into pieces, temporaries as pieces
    bool fused = false;         // levels m-2 and m-1 in one step (the fused short-contraction kernel)
    bool sym = false;           // canonical entries only (in-block symmetry, sym.cuh)
    size_t a_off = 0;
    int state = Q_QUEUED;
    int level = 0;              // next level to launch
    bool split_done = false;
    size_t ws_off = 0, ws_bytes = 0, x_off = 0, buf_off[2] = {0, 0};
    int rows = 0, Kp = 0;
    double t_submit = 0, t_done = 0;
    std::vector<Tile> tiles[STTSM_MAX_M];
    std::vector<TcInst> inst;       // per level (released when the request is done)
    std::vector<TmaInst> tinst;     // per level, TMA-fed requests only
    bool tables_held = false;       // holds a reference on its shape's level tables
};

// Level tables of one shape (m, nbar, b): the G table and offset table of
// every level, one allocation in the table region.
struct TableSet {
    size_t off = 0, bytes = 0;
    size_t level_off[STTSM_MAX_M] = {};
    int refs = 0;
    uint64_t last_use = 0;
};

struct StepRec {
    int ev;                          // index into the handle's event pool
    std::vector<uint64_t> finishing;
};

struct Staging {
    char* h = nullptr;    // pinned
    char* d = nullptr;
    size_t cap = 0;
    cudaEvent_t copied = nullptr;
};

}  // namespace

struct sttsm_serve_s {
    int prec = 0, np = 0, device = 0, sms = 148;
    bool r64 = false;                    // the last level sums in FP64 (R64 precisions)
    size_t queue_cap = 0;
    char* arena_base = nullptr;
    Arena* arena = nullptr;
    cudaStream_t stream = nullptr;
    int* status = nullptr;
    std::thread th;
    std::atomic<bool> stop{false};
    std::mutex mu;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Req> reqs;
    std::vector<uint64_t> active;
    uint64_t next_ticket = 1;
    uint64_t n_submitted = 0, n_admitted = 0, n_completed = 0;
    char* table_base = nullptr;
    Arena* tables = nullptr;
    char* upload_h = nullptr;            // pinned
    cudaEvent_t upload_done = nullptr;
    std::map<std::tuple<int, int64_t, int>, TableSet> G;   // (m, nbar, b) -> tables
    uint64_t use_clock = 0;
    Staging stg[2];
    int cur = 0;
    cudaEvent_t events[SERVE_EVENTS] = {};
    int next_event = 0;
    std::deque<StepRec> inflight;
    int error = 0;
};

namespace {

// The level tables of shape s, built and copied into the table region on first
// use; returns nullptr when the region has no room even after evicting every
// table set no active request holds (the request then waits).
TableSet* acquire_tables(sttsm_serve_s* H, const Shape& s, int* rc)
{
    *rc = STTSM_OK;
    auto key = std::make_tuple(s.m, s.nbar, s.b);
    auto it = H->G.find(key);
    if (it == H->G.end()) {
        std::vector<int32_t> g[STTSM_MAX_M];
        TableSet T;
        size_t bytes = 0;
        for (int d = 0; d < s.m; ++d) {
            build_level_G(s, d, g[d]);
            T.level_off[d] = bytes;
            bytes = up256(bytes + g[d].size() * sizeof(int32_t));
        }
        T.bytes = bytes;
        while (!H->tables->alloc(bytes, &T.off)) {
            // evict the least recently used table set that no request holds
            auto victim = H->G.end();
            for (auto v = H->G.begin(); v != H->G.end(); ++v)
                if (v->second.refs == 0 && (victim == H->G.end() || v->second.last_use < victim->second.last_use))
                    victim = v;
            if (victim == H->G.end()) return nullptr;
            H->tables->release(victim->second.off, victim->second.bytes);
            H->G.erase(victim);
        }
        // upload through the pinned upload buffer (chunks of its size; it is reused
        // once the previous chunk's copy has finished)
        for (int d = 0; d < s.m; ++d) {
            const char* src = (const char*)g[d].data();
            const size_t total = g[d].size() * sizeof(int32_t);
            for (size_t done = 0; done < total;) {
                const size_t n = std::min(total - done, SERVE_UPLOAD_BYTES);
                if (cudaEventSynchronize(H->upload_done) != cudaSuccess) { *rc = STTSM_ERR_CUDA; return nullptr; }
                memcpy(H->upload_h, src + done, n);
                if (cudaMemcpyAsync(H->table_base + T.off + T.level_off[d] + done, H->upload_h, n, cudaMemcpyHostToDevice,
                                    H->stream) != cudaSuccess ||
                    cudaEventRecord(H->upload_done, H->stream) != cudaSuccess) {
                    *rc = STTSM_ERR_CUDA;
                    return nullptr;
                }
                done += n;
            }
        }
        it = H->G.emplace(key, T).first;
    }
    it->second.refs += 1;
    it->second.last_use = ++H->use_clock;
    return &it->second;
}

void release_tables(sttsm_serve_s* H, const Shape& s)
{
    auto it = H->G.find(std::make_tuple(s.m, s.nbar, s.b));
    if (it != H->G.end() && it->second.refs > 0) it->second.refs -= 1;
}

// Staging bytes one request needs at its current level: its descriptor and tiles.
size_t staging_need(const Req& R)
{
    return (R.tma ? sizeof(TmaInst) : sizeof(TcInst)) + R.tiles[R.level].size() * sizeof(Tile) + sizeof(SplitDesc) + 768;
}

// Builds the request's per-level tiles and descriptors once it has a workspace.
int admit(sttsm_serve_s* H, Req& R, const TableSet& T)
{
    const Shape& s = R.s;
    char* base = H->arena_base + R.ws_off;
    CUtensorMap map, xmaps[TMA_NX];
    const int box = R.small ? TC_SMALL_BN : TC_BN;
    if (R.tma) {
        for (int xs = 0; xs < TMA_NX; ++xs)
            if (make_x_tensor_map(&xmaps[xs], base + R.x_off, H->np, R.rows, R.Kp, 32 * (xs + 1)) != STTSM_OK)
                return STTSM_ERR_CUDA;
    } else if (make_x_tensor_map(&map, base + R.x_off, H->np, R.rows, R.Kp, box) != STTSM_OK) {
        return STTSM_ERR_CUDA;
    }
    R.inst.assign(s.m, TcInst());
    if (R.tma) R.tinst.assign(s.m, TmaInst());
    for (int d = 0; d < s.m; ++d) {
        // R64: the gathered kernel sums in FP64 at every level and the TMA kernel at
        // the last one, with tiles of at most 128 columns there
        const int bn = (H->r64 && !R.small && (!R.tma || d == s.m - 1)) ? R64_BN : box;
        if (R.sym)
            build_level_tiles_sym(s, d, TC_BM, bn, 0, R.tiles[d]);
        else
            build_level_tiles(s, d, TC_BM, bn, 0, R.tiles[d], R.tma && tma_order16x8(s, d));
        const int32_t* G = (const int32_t*)(H->table_base + T.off + T.level_off[d]);
        const LevelShape& LS = s.lv[d];
        TcInst& T = R.inst[d];
        memset(&T, 0, sizeof(T));
        T.tmX = map;
        LevelInst& L = T.L;
        L.parent = d == 0 ? (R.tma ? (const void*)(base + R.a_off) : R.d.A) : (const void*)(base + R.buf_off[(d - 1) & 1]);
        L.out = d == s.m - 1 ? R.d.C : (void*)(base + R.buf_off[d & 1]);
        L.sym_full = d == s.m - 1 ? 1 : 0;
        L.out_np = (R.tma && d < s.m - 1) ? H->np : 0;
        L.G = G;
        L.OFF = G + level_G_size(s, d);
        L.X = R.d.X;
        L.m = s.m; L.b = s.b; L.k = LS.k; L.nbar = (int32_t)s.nbar;
        L.n = (int32_t)s.n; L.p = (int32_t)s.p;
        L.R = (int32_t)s.R;
        L.Ktot = (int32_t)(s.nbar * s.b);
        L.bm = s.bm;
        L.P_parent = LS.P_parent;
        L.P_out = LS.P_out;
        L.rows_per_parent = LS.P_out * s.R;
        int64_t bp = 1;
        for (int q = 0; q <= STTSM_MAX_M; ++q) { L.bpow[q] = (int32_t)(bp < ((int64_t)1 << 31) ? bp : 0); bp *= s.b; }
        if (R.fused && d >= s.m - 2) {
            // levels m-2 and m-1 in one launch: the pair units, writing C
            R.tiles[d].clear();
            if (d == s.m - 2) {
                build_pair_tiles(s, 0, R.tiles[d]);
                L.out = R.d.C;
            }
        }
        if (R.tma) {
            TmaInst& M = R.tinst[d];
            memset(&M, 0, sizeof(M));
            for (int xs = 0; xs < TMA_NX; ++xs) M.tmX[xs] = xmaps[xs];
            L.order16x8 = tma_order16x8(s, d) ? 1 : 0;
            if (make_a_tensor_maps(M.tmA, L.parent, LS.nodes_parent * LS.P_parent, H->np, s.b, s.m, LS.k,
                                   L.order16x8 != 0) != STTSM_OK)
                return STTSM_ERR_CUDA;
            M.L = L;
        }
    }
    return STTSM_OK;
}

// One step: the X split of newly admitted requests, then per tile kind one
// level launch over every active request at its current level.
int launch_step(sttsm_serve_s* H)
{
    std::vector<SplitDesc> split;
    int64_t split_blocks = 0;
    std::vector<const Req*> asplit;            // TMA requests whose A is split this step
    // groups: 0 gathered A, 1 small tiles, 2 / 3 TMA writing pieces / C with b a
    // multiple of 32, 4 / 5 the same with b an odd multiple of 16
    // group 6: the fused last two levels of short contractions
    constexpr int NG = 7;
    std::vector<TcInst> insts[3];               // groups 0, 1, 6
    std::vector<TmaInst> tinsts[4];             // groups 2 .. 5
    std::vector<Tile> tiles[NG];
    std::vector<uint64_t> finishing, stepped, waiting;
    size_t need = 0;
    for (uint64_t tk : H->active) {
        Req& R = H->reqs[tk];
        const size_t rn = staging_need(R);
        if (need + rn > SERVE_STAGING_BYTES - SERVE_STAGING_SLACK) { waiting.push_back(tk); continue; }   // next step
        need += rn;
        stepped.push_back(tk);
        if (!R.split_done) {
            SplitDesc sd;
            sd.X = (const float*)R.d.X;
            sd.out = H->arena_base + R.ws_off + R.x_off;
            sd.p = (int)R.d.p; sd.n = (int)R.d.n; sd.rows = R.rows; sd.Kp = R.Kp;
            sd.first_block = split_blocks;
            split_blocks += ((int64_t)R.rows * R.Kp + 255) / 256;
            split.push_back(sd);
            if (R.tma) asplit.push_back(&R);
            R.split_done = true;
        }
        const bool last = R.level == R.s.m - 1;
        const bool pairg = R.fused && R.level == R.s.m - 2;
        const int g = pairg ? 6 : R.tma ? (last ? 3 : 2) + (tma_sw32(R.s) ? 2 : 0) : (R.small ? 1 : 0);
        int32_t e;
        if (g < 2 || g == 6) {
            const int ii = g == 6 ? 2 : g;
            e = (int32_t)insts[ii].size();
            insts[ii].push_back(R.inst[R.level]);
        } else {
            e = (int32_t)tinsts[g - 2].size();
            tinsts[g - 2].push_back(R.tinst[R.level]);
        }
        for (Tile t : R.tiles[R.level]) {
            t.inst = e;
            tiles[g].push_back(t);
        }
    }
    // staging layout: [TmaInst 2..5][TcInst 0, 1][tiles 0..5][split]
    size_t off = 0, o_ti[4], o_i[3], o_t[NG], o_s;
    for (int k = 0; k < 4; ++k) { o_ti[k] = off; off = up256(off + tinsts[k].size() * sizeof(TmaInst)); }
    for (int k = 0; k < 3; ++k) { o_i[k] = off; off = up256(off + insts[k].size() * sizeof(TcInst)); }
    for (int k = 0; k < NG; ++k) { o_t[k] = off; off = up256(off + tiles[k].size() * sizeof(Tile)); }
    o_s = off;
    off = up256(off + split.size() * sizeof(SplitDesc));
    Staging& S = H->stg[H->cur];
    if (off > S.cap) return STTSM_ERR_NOMEM;   // cannot happen: requests were taken while they fit
    // the copy that last read this staging buffer (two steps back) has finished
    if (cudaEventSynchronize(S.copied) != cudaSuccess) return STTSM_ERR_CUDA;
    for (int k = 0; k < 4; ++k)
        if (!tinsts[k].empty()) memcpy(S.h + o_ti[k], tinsts[k].data(), tinsts[k].size() * sizeof(TmaInst));
    for (int k = 0; k < 3; ++k)
        if (!insts[k].empty()) memcpy(S.h + o_i[k], insts[k].data(), insts[k].size() * sizeof(TcInst));
    for (int k = 0; k < NG; ++k)
        if (!tiles[k].empty()) memcpy(S.h + o_t[k], tiles[k].data(), tiles[k].size() * sizeof(Tile));
    if (!split.empty()) memcpy(S.h + o_s, split.data(), split.size() * sizeof(SplitDesc));
    if (cudaMemcpyAsync(S.d, S.h, off, cudaMemcpyHostToDevice, H->stream) != cudaSuccess) return STTSM_ERR_CUDA;
    if (cudaEventRecord(S.copied, H->stream) != cudaSuccess) return STTSM_ERR_CUDA;
    if (!split.empty() &&
        launch_split_x_batch((const SplitDesc*)(S.d + o_s), (int)split.size(), (int)split_blocks, H->np, H->stream) != 0)
        return STTSM_ERR_CUDA;
    for (const Req* R : asplit)
        if (launch_split_bcss((const float*)R->d.A, H->arena_base + R->ws_off + R->a_off, R->s.lv[0].P_parent, R->s.bm,
                              H->np, H->stream) != 0)
            return STTSM_ERR_CUDA;
    TcInst dummy;
    memset(&dummy, 0, sizeof(dummy));
    static TmaInst tdummy;   // zero-initialised; unused when a descriptor table is passed
    for (int k = 0; k < NG; ++k) {
        if (tiles[k].empty()) continue;
        const Tile* dt = (const Tile*)(S.d + o_t[k]);
        const int n = (int)tiles[k].size();
        int lrc;
        int maxc = 0;
        int symf = 0;
        for (const Tile& t : tiles[k]) {
            maxc = std::max(maxc, (int)t.ncols);
            symf |= (t.pad0 & 3) == SYM_TILE ? 1 : 0;
        }
        if (k == 0 && H->r64)
            lrc = launch_level_tc_r64(H->np, dummy, (const TcInst*)(S.d + o_i[0]), dt, n, H->sms, H->status, maxc, H->stream);
        else if (k == 0) lrc = launch_level_tc(H->np, dummy, (const TcInst*)(S.d + o_i[0]), dt, n, H->sms, H->status, H->stream);
        else if (k == 1 && (small_kernel_kind() == 0 || H->r64))
            lrc = launch_level_small_f32_tc((const TcInst*)(S.d + o_i[1]), dt, n, H->sms, H->stream, H->r64 ? 1 : 0,
                                            symf);
        else if (k == 1) lrc = launch_level_tc_small(H->np, dummy, (const TcInst*)(S.d + o_i[1]), dt, n, H->sms, H->status, H->stream);
        else if (k == 6) lrc = launch_level_pair_f32_tc((const TcInst*)(S.d + o_i[2]), dt, n, H->sms, H->stream);
        else {
            const int ck = H->r64 ? TMA_OUT_C64 : TMA_OUT_C;
            lrc = launch_level_tma(H->np, tdummy, (const TmaInst*)(S.d + o_ti[k - 2]), dt, n, H->sms, H->status,
                                   (k & 1) == 1 ? ck : TMA_OUT_PIECES, k >= 4, maxc, H->stream);
        }
        if (lrc != 0) return STTSM_ERR_CUDA;
    }
    H->cur ^= 1;
    // advance the stepped requests by one level (the finished ones wait for this
    // step's event); requests left out of this step go first in the next
    std::vector<uint64_t> still = waiting;
    for (uint64_t tk : stepped) {
        Req& R = H->reqs[tk];
        R.level += (R.fused && R.level == R.s.m - 2) ? 2 : 1;
        if (R.level == R.s.m) {
            R.state = Q_FINISHING;
            finishing.push_back(tk);
        } else {
            still.push_back(tk);
        }
    }
    H->active.swap(still);
    StepRec rec;
    rec.ev = H->next_event;
    H->next_event = (H->next_event + 1) % SERVE_EVENTS;
    if (cudaEventRecord(H->events[rec.ev], H->stream) != cudaSuccess) return STTSM_ERR_CUDA;
    rec.finishing.swap(finishing);
    H->inflight.push_back(std::move(rec));
    return STTSM_OK;
}

void scheduler(sttsm_serve_s* H)
{
    cudaSetDevice(H->device);
    while (!H->stop.load()) {
        bool progress = false;
        // retire completed steps
        while (!H->inflight.empty()) {
            const cudaError_t q = cudaEventQuery(H->events[H->inflight.front().ev]);
            if (q == cudaErrorNotReady) break;
            const double t = now_s();
            std::lock_guard<std::mutex> lock(H->mu);
            if (q != cudaSuccess && !H->error) H->error = STTSM_ERR_CUDA;
            for (uint64_t tk : H->inflight.front().finishing) {
                Req& R = H->reqs[tk];
                R.state = Q_DONE;
                R.t_done = t;
                H->arena->release(R.ws_off, R.ws_bytes);
                if (R.tables_held) { release_tables(H, R.s); R.tables_held = false; }
                for (int d = 0; d < STTSM_MAX_M; ++d) std::vector<Tile>().swap(R.tiles[d]);
                std::vector<TcInst>().swap(R.inst);
                std::vector<TmaInst>().swap(R.tinst);
                ++H->n_completed;
            }
            H->inflight.pop_front();
            progress = true;
        }
        // admission in arrival order; a request whose workspace (or level tables)
        // does not fit yet is passed by later ones until it is older than the age
        // cap, after which nothing passes it
        {
            std::lock_guard<std::mutex> lock(H->mu);
            const double t = now_s();
            int scanned = 0;
            for (auto qi = H->queue.begin(); qi != H->queue.end() && !H->error && scanned < SERVE_PASS_WINDOW;
                 ++scanned) {
                Req& R = H->reqs[*qi];
                size_t off = 0;
                bool ok = H->arena->alloc(R.ws_bytes, &off);
                TableSet* T = nullptr;
                if (ok) {
                    int rc = STTSM_OK;
                    T = acquire_tables(H, R.s, &rc);
                    if (rc != STTSM_OK) { H->error = rc; break; }
                    if (!T) { H->arena->release(off, R.ws_bytes); ok = false; }
                }
                if (!ok) {
                    if (t - R.t_submit > SERVE_AGE_CAP_S) break;   // it waits; nothing passes it
                    ++qi;
                    continue;
                }
                R.ws_off = off;
                R.tables_held = true;
                const int rc = admit(H, R, *T);
                if (rc != STTSM_OK) { H->error = rc; break; }
                R.state = Q_ACTIVE;
                H->active.push_back(*qi);
                qi = H->queue.erase(qi);
                ++H->n_admitted;
                progress = true;
            }
        }
        if (!H->active.empty() && H->inflight.size() < 2 && !H->error) {
            std::lock_guard<std::mutex> lock(H->mu);
            const int rc = launch_step(H);
            if (rc != STTSM_OK) H->error = rc;
            progress = true;
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void destroy(sttsm_serve_s* H)
{
    if (!H) return;
    H->stop.store(true);
    if (H->th.joinable()) H->th.join();
    if (H->stream) cudaStreamSynchronize(H->stream);
    for (cudaEvent_t& e : H->events)
        if (e) cudaEventDestroy(e);
    if (H->table_base) cudaFree(H->table_base);
    delete H->tables;
    if (H->upload_h) cudaFreeHost(H->upload_h);
    if (H->upload_done) cudaEventDestroy(H->upload_done);
    for (Staging& S : H->stg) {
        if (S.h) cudaFreeHost(S.h);
        if (S.d) cudaFree(S.d);
        if (S.copied) cudaEventDestroy(S.copied);
    }
    if (H->arena_base) cudaFree(H->arena_base);
    delete H->arena;
    if (H->stream) cudaStreamDestroy(H->stream);
    delete H;
}

}  // namespace

extern "C" {

int sttsm_serve_create(size_t hbm_budget_bytes, int prec, int queue_cap, void** handle)
{
    if (!handle || hbm_budget_bytes < 256 || queue_cap < 1) return STTSM_ERR_ARG;
    if (prec_npiece(prec) == 0) return STTSM_ERR_UNSUPPORTED;
    sttsm_serve_s* H = new sttsm_serve_s();
    H->prec = prec;
    H->np = prec_npiece(prec);
    H->r64 = prec_r64(prec);
    H->queue_cap = (size_t)queue_cap;
    cudaGetDevice(&H->device);
    if (cudaDeviceGetAttribute(&H->sms, cudaDevAttrMultiProcessorCount, H->device) != cudaSuccess || H->sms <= 0) H->sms = 148;
    H->status = batch_status_word();
    bool ok = H->status && cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc((void**)&H->arena_base, up256(hbm_budget_bytes)) == cudaSuccess &&
              cudaMalloc((void**)&H->table_base, SERVE_TABLE_BYTES) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) {
        Staging& S = H->stg[k];
        ok = cudaHostAlloc((void**)&S.h, SERVE_STAGING_BYTES, cudaHostAllocDefault) == cudaSuccess &&
             cudaMalloc((void**)&S.d, SERVE_STAGING_BYTES) == cudaSuccess &&
             cudaEventCreateWithFlags(&S.copied, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventRecord(S.copied, H->stream) == cudaSuccess;
        if (ok) S.cap = SERVE_STAGING_BYTES;
    }
    for (int k = 0; k < SERVE_EVENTS && ok; ++k)
        ok = cudaEventCreateWithFlags(&H->events[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaHostAlloc((void**)&H->upload_h, SERVE_UPLOAD_BYTES, cudaHostAllocDefault) == cudaSuccess &&
         cudaEventCreateWithFlags(&H->upload_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventRecord(H->upload_done, H->stream) == cudaSuccess;
    if (!ok) {
        destroy(H);
        return STTSM_ERR_NOMEM;
    }
    H->arena = new Arena(up256(hbm_budget_bytes));
    H->tables = new Arena(SERVE_TABLE_BYTES);
    H->th = std::thread(scheduler, H);
    *handle = H;
    return STTSM_OK;
}

int sttsm_serve_submit(void* h, const sttsm_desc* d, uint64_t* ticket)
{
    sttsm_serve_s* H = (sttsm_serve_s*)h;
    if (!H || !d || !ticket || !d->A || !d->X || !d->C) return STTSM_ERR_ARG;
    if (((uintptr_t)d->A | (uintptr_t)d->X | (uintptr_t)d->C) % 16 != 0) return STTSM_ERR_ARG;
    if (d->n >= ((int64_t)1 << 30) || d->p >= ((int64_t)1 << 30)) return STTSM_ERR_UNSUPPORTED;
    Req R;
    R.d = *d;
    int rc = make_shape(d->m, d->n, d->p, d->b, &R.s);
    if (rc != STTSM_OK) return rc;
    R.small = tc_small_mode(R.s);
    R.tma = tc_tma_mode(R.s);
    R.sym = sym_levels(R.s, H->prec);
    R.fused = R.small && !H->r64 && small_kernel_kind() == 0 && fused_tail_in_batches() && pair_mode(R.s) && !R.sym;
    R.rows = (int)(R.s.pbar * R.s.b);
    R.Kp = (int)(((R.s.nbar * R.s.b) + 7) / 8 * 8);
    R.x_off = 0;
    const size_t esz = R.tma ? 2 * (size_t)H->np : 4;
    size_t off = up256((size_t)H->np * R.rows * R.Kp * 2);
    R.a_off = off;
    if (R.tma) off += up256((size_t)H->np * R.s.lv[0].P_parent * R.s.bm * 2);
    R.buf_off[0] = off;
    off += up256((size_t)R.s.buf_elems[0] * esz);
    R.buf_off[1] = off;
    off += up256((size_t)R.s.buf_elems[1] * esz);
    R.ws_bytes = std::max<size_t>(off, 256);
    // a request must fit one step's staging buffer at every level
    for (int lv = 0; lv < R.s.m; ++lv)
        if (level_tile_count(R.s, lv, TC_BM, R.small ? TC_SMALL_BN : TC_BN) * sizeof(Tile) + sizeof(TmaInst) + 1024 >
            SERVE_STAGING_BYTES - SERVE_STAGING_SLACK)
            return STTSM_ERR_NOMEM;
    std::lock_guard<std::mutex> lock(H->mu);
    if (H->error) return H->error;
    if (R.ws_bytes > H->arena->size()) return STTSM_ERR_NOMEM;
    if (H->queue.size() >= H->queue_cap) return STTSM_ERR_BUSY;
    R.t_submit = now_s();
    const uint64_t tk = H->next_ticket++;
    H->reqs.emplace(tk, std::move(R));
    H->queue.push_back(tk);
    ++H->n_submitted;
    *ticket = tk;
    return STTSM_OK;
}

int sttsm_serve_poll(void* h, uint64_t ticket, int* done, double* latency_ms)
{
    sttsm_serve_s* H = (sttsm_serve_s*)h;
    if (!H || !done) return STTSM_ERR_ARG;
    std::lock_guard<std::mutex> lock(H->mu);
    auto it = H->reqs.find(ticket);
    if (it == H->reqs.end()) return STTSM_ERR_ARG;
    *done = it->second.state == Q_DONE ? 1 : 0;
    if (latency_ms) *latency_ms = *done ? (it->second.t_done - it->second.t_submit) * 1e3 : -1.0;
    if (H->error) return H->error;
    return peek_status_word() != 0 ? STTSM_ERR_TIMEOUT : STTSM_OK;
}

int sttsm_serve_stats(void* h, uint64_t* out)
{
    sttsm_serve_s* H = (sttsm_serve_s*)h;
    if (!H || !out) return STTSM_ERR_ARG;
    std::lock_guard<std::mutex> lock(H->mu);
    out[0] = H->n_submitted;
    out[1] = H->n_admitted;
    out[2] = H->n_completed;
    out[3] = H->queue.size();
    out[4] = H->active.size();
    out[5] = H->arena->used();
    return STTSM_OK;
}

int sttsm_serve_destroy(void* h)
{
    destroy((sttsm_serve_s*)h);
    return STTSM_OK;
}

}  // extern "C"
