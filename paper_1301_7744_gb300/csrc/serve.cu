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
#include "sttsm.h"

using namespace sttsm;

namespace sttsm {
int* batch_status_word();   // capi.cu
int peek_status_word();     // capi.cu
}

namespace {

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

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
};

struct StepRec {
    cudaEvent_t ev;
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
    std::map<std::tuple<int, int64_t, int, int>, std::pair<int32_t*, std::vector<int32_t>>> G;
    Staging stg[2];
    int cur = 0;
    std::deque<StepRec> inflight;
    int error = 0;
};

namespace {

int ensure_G(sttsm_serve_s* H, const Shape& s, int d, const int32_t** out)
{
    auto key = std::make_tuple(s.m, s.nbar, s.b, d);
    auto it = H->G.find(key);
    if (it == H->G.end()) {
        std::vector<int32_t> g;
        build_level_G(s, d, g);
        int32_t* dg = nullptr;
        if (cudaMalloc(&dg, g.size() * sizeof(int32_t)) != cudaSuccess) return STTSM_ERR_NOMEM;
        it = H->G.emplace(key, std::make_pair(dg, std::move(g))).first;
        if (cudaMemcpyAsync(dg, it->second.second.data(), it->second.second.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, H->stream) != cudaSuccess)
            return STTSM_ERR_CUDA;
    }
    *out = it->second.first;
    return STTSM_OK;
}

// Builds the request's per-level tiles and descriptors once it has a workspace.
int admit(sttsm_serve_s* H, Req& R)
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
        build_level_tiles(s, d, TC_BM, box, 0, R.tiles[d]);
        const int32_t* G = nullptr;
        const int rc = ensure_G(H, s, d, &G);
        if (rc != STTSM_OK) return rc;
        const LevelShape& LS = s.lv[d];
        TcInst& T = R.inst[d];
        memset(&T, 0, sizeof(T));
        T.tmX = map;
        LevelInst& L = T.L;
        L.parent = d == 0 ? (R.tma ? (const void*)(base + R.a_off) : R.d.A) : (const void*)(base + R.buf_off[(d - 1) & 1]);
        L.out = d == s.m - 1 ? R.d.C : (void*)(base + R.buf_off[d & 1]);
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
        if (R.tma) {
            TmaInst& M = R.tinst[d];
            memset(&M, 0, sizeof(M));
            for (int xs = 0; xs < TMA_NX; ++xs) M.tmX[xs] = xmaps[xs];
            if (make_a_tensor_maps(M.tmA, L.parent, LS.nodes_parent * LS.P_parent, H->np, s.b, s.m, LS.k) != STTSM_OK)
                return STTSM_ERR_CUDA;
            M.L = L;
        }
    }
    return STTSM_OK;
}

int grow_staging(sttsm_serve_s* H, Staging& S, size_t need)
{
    if (S.cap >= need) return STTSM_OK;
    if (cudaStreamSynchronize(H->stream) != cudaSuccess) return STTSM_ERR_CUDA;
    if (S.h) cudaFreeHost(S.h);
    if (S.d) cudaFree(S.d);
    S.h = nullptr; S.d = nullptr; S.cap = 0;
    const size_t cap = std::max(need + need / 2, (size_t)1 << 20);
    if (cudaHostAlloc((void**)&S.h, cap, cudaHostAllocDefault) != cudaSuccess) return STTSM_ERR_NOMEM;
    if (cudaMalloc((void**)&S.d, cap) != cudaSuccess) return STTSM_ERR_NOMEM;
    S.cap = cap;
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
    constexpr int NG = 6;
    std::vector<TcInst> insts[2];
    std::vector<TmaInst> tinsts[NG - 2];
    std::vector<Tile> tiles[NG];
    std::vector<uint64_t> finishing;
    for (uint64_t tk : H->active) {
        Req& R = H->reqs[tk];
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
        const int g = R.tma ? (last ? 3 : 2) + (tma_sw32(R.s) ? 2 : 0) : (R.small ? 1 : 0);
        int32_t e;
        if (g < 2) { e = (int32_t)insts[g].size(); insts[g].push_back(R.inst[R.level]); }
        else { e = (int32_t)tinsts[g - 2].size(); tinsts[g - 2].push_back(R.tinst[R.level]); }
        for (Tile t : R.tiles[R.level]) {
            t.inst = e;
            tiles[g].push_back(t);
        }
    }
    // staging layout: [TmaInst 2..5][TcInst 0, 1][tiles 0..5][split]
    size_t off = 0, o_ti[NG - 2], o_i[2], o_t[NG], o_s;
    for (int k = 0; k < NG - 2; ++k) { o_ti[k] = off; off = up256(off + tinsts[k].size() * sizeof(TmaInst)); }
    for (int k = 0; k < 2; ++k) { o_i[k] = off; off = up256(off + insts[k].size() * sizeof(TcInst)); }
    for (int k = 0; k < NG; ++k) { o_t[k] = off; off = up256(off + tiles[k].size() * sizeof(Tile)); }
    o_s = off;
    off = up256(off + split.size() * sizeof(SplitDesc));
    Staging& S = H->stg[H->cur];
    if (S.copied && cudaEventSynchronize(S.copied) != cudaSuccess) return STTSM_ERR_CUDA;
    int rc = grow_staging(H, S, off);
    if (rc != STTSM_OK) return rc;
    if (!S.copied && cudaEventCreateWithFlags(&S.copied, cudaEventDisableTiming) != cudaSuccess) return STTSM_ERR_CUDA;
    for (int k = 0; k < NG - 2; ++k)
        if (!tinsts[k].empty()) memcpy(S.h + o_ti[k], tinsts[k].data(), tinsts[k].size() * sizeof(TmaInst));
    for (int k = 0; k < 2; ++k)
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
        if (k == 0) lrc = launch_level_tc(H->np, dummy, (const TcInst*)(S.d + o_i[0]), dt, n, H->sms, H->status, H->stream);
        else if (k == 1 && small_kernel_kind() == 0) lrc = launch_level_small_f32_tc((const TcInst*)(S.d + o_i[1]), dt, n, H->sms, H->stream);
        else if (k == 1) lrc = launch_level_tc_small(H->np, dummy, (const TcInst*)(S.d + o_i[1]), dt, n, H->sms, H->status, H->stream);
        else {
            int maxc = 0;
            for (const Tile& t : tiles[k]) maxc = std::max(maxc, (int)t.ncols);
            lrc = launch_level_tma(H->np, tdummy, (const TmaInst*)(S.d + o_ti[k - 2]), dt, n, H->sms, H->status,
                                   (k & 1) == 1 ? TMA_OUT_C : TMA_OUT_PIECES, k >= 4, maxc, H->stream);
        }
        if (lrc != 0) return STTSM_ERR_CUDA;
    }
    H->cur ^= 1;
    // advance every request by one level; the finished ones wait for this step's event
    std::vector<uint64_t> still;
    for (uint64_t tk : H->active) {
        Req& R = H->reqs[tk];
        if (++R.level == R.s.m) {
            R.state = Q_FINISHING;
            finishing.push_back(tk);
        } else {
            still.push_back(tk);
        }
    }
    H->active.swap(still);
    StepRec rec;
    if (cudaEventCreateWithFlags(&rec.ev, cudaEventDisableTiming) != cudaSuccess) return STTSM_ERR_CUDA;
    if (cudaEventRecord(rec.ev, H->stream) != cudaSuccess) return STTSM_ERR_CUDA;
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
            const cudaError_t q = cudaEventQuery(H->inflight.front().ev);
            if (q == cudaErrorNotReady) break;
            const double t = now_s();
            std::lock_guard<std::mutex> lock(H->mu);
            if (q != cudaSuccess && !H->error) H->error = STTSM_ERR_CUDA;
            for (uint64_t tk : H->inflight.front().finishing) {
                Req& R = H->reqs[tk];
                R.state = Q_DONE;
                R.t_done = t;
                H->arena->release(R.ws_off, R.ws_bytes);
                for (int d = 0; d < STTSM_MAX_M; ++d) std::vector<Tile>().swap(R.tiles[d]);
                std::vector<TcInst>().swap(R.inst);
                std::vector<TmaInst>().swap(R.tinst);
                ++H->n_completed;
            }
            cudaEventDestroy(H->inflight.front().ev);
            H->inflight.pop_front();
            progress = true;
        }
        // admission in arrival order while the workspace fits
        {
            std::lock_guard<std::mutex> lock(H->mu);
            while (!H->queue.empty() && !H->error) {
                Req& R = H->reqs[H->queue.front()];
                size_t off = 0;
                if (!H->arena->alloc(R.ws_bytes, &off)) break;
                R.ws_off = off;
                const int rc = admit(H, R);
                if (rc != STTSM_OK) { H->error = rc; break; }
                R.state = Q_ACTIVE;
                H->active.push_back(H->queue.front());
                H->queue.pop_front();
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
    for (auto& r : H->inflight) cudaEventDestroy(r.ev);
    for (auto& kv : H->G) cudaFree(kv.second.first);
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
    if (prec != STTSM_BF16X6 && prec != STTSM_BF16X3) return STTSM_ERR_UNSUPPORTED;
    sttsm_serve_s* H = new sttsm_serve_s();
    H->prec = prec;
    H->np = prec == STTSM_BF16X6 ? 3 : 2;
    H->queue_cap = (size_t)queue_cap;
    cudaGetDevice(&H->device);
    if (cudaDeviceGetAttribute(&H->sms, cudaDevAttrMultiProcessorCount, H->device) != cudaSuccess || H->sms <= 0) H->sms = 148;
    H->status = batch_status_word();
    if (!H->status || cudaStreamCreateWithFlags(&H->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc((void**)&H->arena_base, up256(hbm_budget_bytes)) != cudaSuccess) {
        destroy(H);
        return STTSM_ERR_NOMEM;
    }
    H->arena = new Arena(up256(hbm_budget_bytes));
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
