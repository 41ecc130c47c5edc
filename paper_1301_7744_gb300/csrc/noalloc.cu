// noalloc.cu — sttsm_bcss_noalloc: the sttsm_bcss computation for callers
// that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc (or any allocator) at the
// point where they run sttsm: code running under a fixed, pre-reserved memory
// budget (embedded and real-time services), plug-ins hosted by a framework
// that owns every device allocation, and paths where an allocation could
// stall or fail at an unpredictable moment.  This entry point needs nothing
// from them but the inputs and the output: its workspace (the split X pieces,
// the ping-pong buffers of the temporaries and the level plans) lives in one
// file-scope device array of STTSM_NOALLOC_SCRATCH_BYTES bytes, which every
// GPU that loads the library holds until the process exits.
//
// Host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress while that device is current and
// caches it.  The same first call page-locks and maps a static host word per
// device (cudaHostRegister, no allocation) that the kernels raise when a
// bounded wait runs out; every later call reads and clears it before it
// launches and then returns STTSM_ERR_TIMEOUT, as sttsm_bcss does with its own
// status word.  Make that first call before any stream capture.
//
// Every call shares the array and finds the previous call's contents there:
// nothing in it has to start at zero; the level plans are rebuilt on the
// host and copied in only when the shape or precision changes (the host copy
// is cached with them).  Calls that overlap on the GPU (other streams, other
// host threads) race on the array and corrupt each other's results: serialise
// them.
#include <cstring>
#include <mutex>
#include <vector>
#include "launch.h"
#include "plan.h"
#include "sttsm.h"

using namespace sttsm;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[STTSM_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
constexpr int STATUS_STRIDE = 16;   // one 64-byte line per device

// Host status words, one per device; page-locked and mapped at set-up.  The
// array spans whole 64 KiB pages (the largest host page size in use), so the
// registration pins nothing else.
alignas(65536) int g_status_host[65536 / sizeof(int)];

struct DevScratch {
    unsigned char* base = nullptr;   // device address of g_noalloc_scratch
    int* status = nullptr;           // device address of this device's host status word
    // plans resident in the array, and their host copy
    int m = 0, b = 0, prec = -1;
    int64_t n = 0, p = 0;
    std::vector<Tile> tiles[STTSM_MAX_M];
    std::vector<int32_t> G[STTSM_MAX_M];
};

std::mutex g_mu;
bool g_registered = false;
DevScratch g_dev[MAX_DEVICES];

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

inline volatile int* host_word(int dev) { return (volatile int*)&g_status_host[dev * STATUS_STRIDE]; }

// One-time set-up of device `dev` (current): the scratch array's address and
// the mapped status word.  Called with g_mu held.
int setup_locked(int dev)
{
    DevScratch& D = g_dev[dev];
    if (D.base) return STTSM_OK;
    if (!g_registered) {
        if (cudaHostRegister(g_status_host, sizeof(g_status_host), cudaHostRegisterPortable | cudaHostRegisterMapped) !=
            cudaSuccess)
            return STTSM_ERR_CUDA;
        g_registered = true;
    }
    void* st = nullptr;
    if (cudaHostGetDevicePointer(&st, (void*)host_word(dev), 0) != cudaSuccess || !st) return STTSM_ERR_CUDA;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return STTSM_ERR_CUDA;
    *host_word(dev) = 0;
    D.status = (int*)st;
    D.base = (unsigned char*)ptr;
    return STTSM_OK;
}

int current_device(int* dev)
{
    if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= MAX_DEVICES) return STTSM_ERR_CUDA;
    return STTSM_OK;
}

}  // namespace

extern "C" int sttsm_bcss_noalloc(const void* A, const void* X, int m, int64_t n, int64_t p, int b, void* C,
                                  int prec, void* stream_)
{
    if (!A || !X || !C) return STTSM_ERR_ARG;
    if (prec == STTSM_TF32X3) return STTSM_ERR_UNSUPPORTED;
    if (prec_r64(prec)) return STTSM_ERR_UNSUPPORTED;
    if (prec != STTSM_FP64 && prec != STTSM_BF16X6 && prec != STTSM_BF16X3) return STTSM_ERR_ARG;
    if (((uintptr_t)A | (uintptr_t)X | (uintptr_t)C) % 16 != 0) return STTSM_ERR_ARG;
    if (n >= (int64_t)1 << 30 || p >= (int64_t)1 << 30) return STTSM_ERR_UNSUPPORTED;
    Shape s;
    int rc = make_shape(m, n, p, b, &s);
    if (rc != STTSM_OK) return rc;
    int dev = 0;
    if ((rc = current_device(&dev)) != STTSM_OK) return rc;
    cudaStream_t stream = (cudaStream_t)stream_;

    const bool fp64 = prec == STTSM_FP64;
    const bool small = !fp64 && tc_small_mode(s);
    const int BM = fp64 ? 64 : TC_BM, BN = fp64 ? 64 : (small ? TC_SMALL_BN : TC_BN);
    const int np = prec == STTSM_BF16X6 ? 3 : (prec == STTSM_BF16X3 ? 2 : 0);
    const size_t esz = fp64 ? 8 : 4;
    const int rows = (int)(s.pbar * s.b), Kp = (int)(((s.nbar * s.b) + 7) / 8 * 8);

    std::lock_guard<std::mutex> lock(g_mu);
    if ((rc = setup_locked(dev)) != STTSM_OK) return rc;
    DevScratch& D = g_dev[dev];
    // a bounded wait of an earlier call ran out: report it once
    if (__atomic_exchange_n((int*)host_word(dev), 0, __ATOMIC_SEQ_CST) != 0) return STTSM_ERR_TIMEOUT;

    // level plans on the host: rebuilt only when the shape or precision changes
    const bool same = D.m == m && D.n == n && D.p == p && D.b == b && D.prec == prec;
    std::vector<Tile> tiles_new[STTSM_MAX_M];
    std::vector<int32_t> G_new[STTSM_MAX_M];
    const std::vector<Tile>* tiles = D.tiles;
    const std::vector<int32_t>* G = D.G;
    if (!same) {
        for (int d = 0; d < m; ++d) {
            build_level_tiles(s, d, BM, BN, 0, tiles_new[d]);
            build_level_G(s, d, G_new[d]);
        }
        tiles = tiles_new;
        G = G_new;
    }

    // layout of the array: [tiles per level][G per level][X pieces][buffer 0][buffer 1]
    size_t off = 0;
    size_t tiles_off[STTSM_MAX_M], G_off[STTSM_MAX_M];
    for (int d = 0; d < m; ++d) { tiles_off[d] = off; off = up256(off + tiles[d].size() * sizeof(Tile)); }
    for (int d = 0; d < m; ++d) { G_off[d] = off; off = up256(off + G[d].size() * sizeof(int32_t)); }
    const size_t x_off = off;
    off = up256(off + (size_t)np * rows * Kp * 2);
    const size_t buf_off[2] = {off, up256(off + (size_t)s.buf_elems[0] * esz)};
    const size_t total = up256(buf_off[1] + (size_t)s.buf_elems[1] * esz);
    if (total > (size_t)STTSM_NOALLOC_SCRATCH_BYTES) return STTSM_ERR_NOMEM;

    unsigned char* base = D.base;
    if (!same) {
        // a copy recorded into a capturing stream would run later, from host
        // memory that the next shape change overwrites: refuse it
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return STTSM_ERR_CUDA;
        if (cap != cudaStreamCaptureStatusNone) return STTSM_ERR_UNSUPPORTED;
        D.prec = -1;   // the resident plans are being replaced
        for (int d = 0; d < STTSM_MAX_M; ++d) {
            D.tiles[d].swap(tiles_new[d]);
            D.G[d].swap(G_new[d]);
        }
        tiles = D.tiles;
        G = D.G;
        for (int d = 0; d < m; ++d) {
            if (cudaMemcpyAsync(base + tiles_off[d], tiles[d].data(), tiles[d].size() * sizeof(Tile),
                                cudaMemcpyHostToDevice, stream) != cudaSuccess ||
                cudaMemcpyAsync(base + G_off[d], G[d].data(), G[d].size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, stream) != cudaSuccess)
                return STTSM_ERR_CUDA;
        }
        D.m = m; D.n = n; D.p = p; D.b = b; D.prec = prec;
    }

    int* status = D.status;
    void* bufs[2] = {base + buf_off[0], base + buf_off[1]};
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    TcInst ti;
    memset(&ti, 0, sizeof(ti));
    if (!fp64) {
        if (launch_split_x((const float*)X, base + x_off, (int)p, (int)n, rows, Kp, np, stream) != 0) return STTSM_ERR_CUDA;
        if (make_x_tensor_map(&ti.tmX, base + x_off, np, rows, Kp, BN) != STTSM_OK) return STTSM_ERR_CUDA;
    }
    for (int d = 0; d < m; ++d) {
        const LevelShape& LS = s.lv[d];
        LevelInst& L = ti.L;
        L.parent = d == 0 ? A : bufs[(d - 1) & 1];
        L.out = d == m - 1 ? C : bufs[d & 1];
        L.G = (const int32_t*)(base + G_off[d]);
        L.OFF = L.G + level_G_size(s, d);
        L.X = X;
        L.m = m; L.b = b; L.k = LS.k; L.nbar = (int32_t)s.nbar;
        L.n = (int32_t)n; L.p = (int32_t)p;
        L.R = (int32_t)s.R;
        L.Ktot = (int32_t)(s.nbar * b);
        L.bm = s.bm;
        L.P_parent = LS.P_parent;
        L.P_out = LS.P_out;
        L.rows_per_parent = LS.P_out * s.R;
        int64_t bp = 1;
        for (int a = 0; a <= STTSM_MAX_M; ++a) { L.bpow[a] = (int32_t)(bp < ((int64_t)1 << 31) ? bp : 0); bp *= b; }
        const Tile* dt = (const Tile*)(base + tiles_off[d]);
        const int nt = (int)tiles[d].size();
        int lrc = fp64 ? launch_level_fp64(L, nullptr, dt, nt, sms, stream)
                  : (small && small_kernel_kind() == 0) ? launch_level_small_f32(L, nullptr, dt, nt, sms, stream)
                  : small ? launch_level_tc_small(np, ti, nullptr, dt, nt, sms, status, stream)
                          : launch_level_tc(np, ti, nullptr, dt, nt, sms, status, stream);
        if (lrc != 0) return STTSM_ERR_CUDA;
    }
    return STTSM_OK;
}

// Runs the bounded-wait probe on this entry point's status word (set up on the
// current device if needed) and synchronises the device; the status is left
// for the next sttsm_bcss_noalloc call to report.
extern "C" int sttsm_noalloc_selftest_wait_timeout(double limit_ms)
{
    if (!(limit_ms > 0.0) || limit_ms > 1000.0) return STTSM_ERR_ARG;
    int dev = 0, rc;
    if ((rc = current_device(&dev)) != STTSM_OK) return rc;
    int* status = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if ((rc = setup_locked(dev)) != STTSM_OK) return rc;
        status = g_dev[dev].status;
    }
    if (launch_wait_probe(status, (unsigned long long)(limit_ms * 1e6), nullptr) != 0) return STTSM_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return STTSM_ERR_CUDA;
    return STTSM_OK;
}
