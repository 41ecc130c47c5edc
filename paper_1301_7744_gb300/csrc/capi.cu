// capi.cu — C ABI of the sttsm library (declared in include/sttsm.h).
#include <cudaTypedefs.h>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>
#include "launch.h"
#include "plan.h"
#include "sym.cuh"
#include "sttsm.h"

using namespace sttsm;

namespace {

int* g_status_host = nullptr;   // host-mapped pinned status word
int* g_status_dev = nullptr;
std::mutex g_status_mu;

int* status_dev()
{
    std::lock_guard<std::mutex> lock(g_status_mu);
    if (!g_status_host) {
        if (cudaHostAlloc((void**)&g_status_host, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess)
            return nullptr;
        *g_status_host = 0;
        if (cudaHostGetDevicePointer((void**)&g_status_dev, g_status_host, 0) != cudaSuccess) return nullptr;
    }
    return g_status_dev;
}

int take_status()
{
    if (!g_status_host) return 0;
    int v = __atomic_exchange_n(g_status_host, 0, __ATOMIC_SEQ_CST);
    return v;
}

int num_sms()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    return v;
}

// ---- per-launch event timing (sttsm_profile_*)
struct ProfRec {
    cudaEvent_t a, b;
    int kind, level;
    double flops;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;

struct ProfScope {
    cudaStream_t s;
    ProfRec r;
    bool on;
    ProfScope(cudaStream_t s_, int kind, int level, double flops) : s(s_), on(false)
    {
        std::lock_guard<std::mutex> lock(g_prof_mu);
        if (!g_prof_on) return;
        r.kind = kind; r.level = level; r.flops = flops;
        if (cudaEventCreate(&r.a) != cudaSuccess) return;
        if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return; }
        cudaEventRecord(r.a, s);
        on = true;
    }
    ~ProfScope()
    {
        if (!on) return;
        cudaEventRecord(r.b, s);
        std::lock_guard<std::mutex> lock(g_prof_mu);
        g_prof.push_back(r);
    }
};

void prof_clear_locked()
{
    for (auto& r : g_prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    g_prof.clear();
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int npiece_of(int prec) { return prec_npiece(prec); }

// Workspace layout: [X pieces (split precisions)][A pieces (TMA-fed kernel)]
// [temporaries buffer 0][buffer 1]; the TMA-fed kernel keeps temporaries as
// NP BF16 pieces per entry, the other paths as FP32 / FP64.
struct WsLayout {
    size_t xpieces, apieces, buf0, buf1, total;
    int rows, Kp;
    bool tma;
};

WsLayout ws_layout(const Shape& s, int prec)
{
    WsLayout w;
    const int np = npiece_of(prec);
    w.tma = np && tc_tma_mode(s);
    const size_t esz = prec == STTSM_FP64 ? 8 : (w.tma ? 2 * (size_t)np : 4);
    w.rows = (int)(s.pbar * s.b);
    w.Kp = (int)(((s.nbar * s.b) + 7) / 8 * 8);
    w.xpieces = 0;
    size_t off = np ? align256((size_t)np * w.rows * w.Kp * 2) : 0;
    w.apieces = off;
    if (w.tma) off += align256((size_t)np * s.lv[0].P_parent * s.bm * 2);
    w.buf0 = off;
    off += align256((size_t)s.buf_elems[0] * esz);
    w.buf1 = off;
    off += align256((size_t)s.buf_elems[1] * esz);
    w.total = off;
    return w;
}

int cuda_err(int e) { return e == 0 ? STTSM_OK : STTSM_ERR_CUDA; }

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

}  // namespace

namespace sttsm {

std::atomic<int> g_small_kind{0};
int small_kernel_kind() { return g_small_kind.load(); }
std::atomic<int> g_fused_tail{1};
bool fused_tail_enabled() { return g_fused_tail.load() != 0; }
bool fused_tail_in_batches() { return g_fused_tail.load() == 2; }
std::atomic<int> g_inblock_sym{0};
bool inblock_sym_enabled() { return g_inblock_sym.load() != 0; }
bool sym_levels(const Shape& s, int prec)
{
    return inblock_sym_enabled() && prec_npiece(prec) > 0 && tc_small_mode(s) &&
           (small_kernel_kind() == 0 || prec_r64(prec)) && sym_shape_ok(s);
}

int* batch_status_word() { return status_dev(); }
int peek_status_word() { return g_status_host ? __atomic_load_n(g_status_host, __ATOMIC_SEQ_CST) : 0; }

int make_a_tensor_maps(CUtensorMap* maps, const void* pieces, int64_t nblocks, int npiece, int b, int m, int k,
                       bool order16x8)
{
    auto enc = get_encode_fn();
    if (!enc) return STTSM_ERR_CUDA;
    int64_t R = 1;
    for (int a = 0; a < m - 1; ++a) R *= b;
    const int64_t bm = R * b;
    int64_t bq = 1;
    if (order16x8) {
        // tiles of 16 fastest x 8 next rows (m = 3, 4): one 5-D box per 16-wide slice,
        // dims {contraction a, f, r1, r2, block x piece} for q = 0 and {f, a, r1, r2, ...}
        // for q >= 1, where the row modes f, r1, r2 sit at stored position t (t < q) or
        // t + 1 and the contraction at position q
        auto bpow = [&](int e) { int64_t v = 1; for (int i = 0; i < e; ++i) v *= b; return v; };
        for (int q = 0; q <= k; ++q) {
            auto pos = [&](int t) { return t < q ? t : t + 1; };
            const cuuint64_t r2ext = m == 4 ? (cuuint64_t)b : 1;
            const cuuint64_t r2str = (cuuint64_t)(m == 4 ? bpow(pos(2)) : bm) * 2;
            cuuint64_t dims[5] = {(cuuint64_t)b, (cuuint64_t)b, (cuuint64_t)b, r2ext, (cuuint64_t)(nblocks * npiece)};
            cuuint64_t strides[4];
            if (q == 0) {
                strides[0] = (cuuint64_t)bpow(pos(0)) * 2;   // f
            } else {
                strides[0] = (cuuint64_t)bpow(q) * 2;        // contraction
            }
            strides[1] = (cuuint64_t)bpow(pos(1)) * 2;       // r1
            strides[2] = r2str;                               // r2
            strides[3] = (cuuint64_t)bm * 2;                  // block x piece
            cuuint32_t box[5] = {16, 16, 8, 1, (cuuint32_t)npiece};
            cuuint32_t estr[5] = {1, 1, 1, 1, 1};
            const CUresult r = enc(&maps[q], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(pieces), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return STTSM_ERR_CUDA;
        }
        return STTSM_OK;
    }
    if (tma_sw32_b(b)) {
        // one box per 16-wide K slice, 32-byte swizzle
        for (int q = 0; q <= k; ++q, bq *= b) {
            CUresult r;
            if (q == 0) {
                // K-major: {a (contiguous), rows (b apart), block x piece}
                cuuint64_t dims[3] = {(cuuint64_t)b, (cuuint64_t)R, (cuuint64_t)(nblocks * npiece)};
                cuuint64_t strides[2] = {(cuuint64_t)b * 2, (cuuint64_t)bm * 2};
                cuuint32_t box[3] = {16, 128, (cuuint32_t)npiece};
                cuuint32_t estr[3] = {1, 1, 1};
                r = enc(&maps[0], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(pieces), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            } else {
                // MN-major: {16 rows (contiguous), a (b^q apart), 16-row atoms, outer rows (b^(q+1) apart), block x piece};
                // a run of b^q rows that neither divides 128 nor is a multiple of it is
                // loaded one 16-row atom per box (the kernel's atom-by-atom layout)
                const bool atomwise = (bq % 128) != 0 && (128 % bq) != 0;
                cuuint64_t dims[5] = {16, (cuuint64_t)b, (cuuint64_t)(bq / 16), (cuuint64_t)(R / bq),
                                      (cuuint64_t)(nblocks * npiece)};
                cuuint64_t strides[4] = {(cuuint64_t)bq * 2, 32, (cuuint64_t)bq * b * 2, (cuuint64_t)bm * 2};
                cuuint32_t box[5] = {16, 16, atomwise ? 1u : (cuuint32_t)((bq < 128 ? bq : 128) / 16),
                                     atomwise ? 1u : (cuuint32_t)(bq < 128 ? 128 / bq : 1), (cuuint32_t)npiece};
                cuuint32_t estr[5] = {1, 1, 1, 1, 1};
                r = enc(&maps[q], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(pieces), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            }
            if (r != CUDA_SUCCESS) return STTSM_ERR_CUDA;
        }
        return STTSM_OK;
    }
    for (int q = 0; q <= k; ++q, bq *= b) {
        CUresult r;
        if (q == 0) {
            // K-major: {a (contiguous), rows (b apart), block x piece}
            cuuint64_t dims[3] = {(cuuint64_t)b, (cuuint64_t)R, (cuuint64_t)(nblocks * npiece)};
            cuuint64_t strides[2] = {(cuuint64_t)b * 2, (cuuint64_t)bm * 2};
            cuuint32_t box[3] = {32, 128, (cuuint32_t)npiece};
            cuuint32_t estr[3] = {1, 1, 1};
            r = enc(&maps[0], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(pieces), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        } else {
            // MN-major: {32 rows (contiguous), a (b^q apart), 32-row atoms, outer rows (b^(q+1) apart), block x piece}
            cuuint64_t dims[5] = {32, (cuuint64_t)b, (cuuint64_t)(bq / 32), (cuuint64_t)(R / bq), (cuuint64_t)(nblocks * npiece)};
            cuuint64_t strides[4] = {(cuuint64_t)bq * 2, 64, (cuuint64_t)bq * b * 2, (cuuint64_t)bm * 2};
            cuuint32_t box[5] = {32, 32, (cuuint32_t)((bq < 128 ? bq : 128) / 32), (cuuint32_t)(bq < 128 ? 128 / bq : 1),
                                 (cuuint32_t)npiece};
            cuuint32_t estr[5] = {1, 1, 1, 1, 1};
            r = enc(&maps[q], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(pieces), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
        if (r != CUDA_SUCCESS) return STTSM_ERR_CUDA;
    }
    return STTSM_OK;
}

int make_x_tensor_map(CUtensorMap* map, const void* xpieces, int npiece, int rows, int Kp, int box_rows)
{
    auto enc = get_encode_fn();
    if (!enc) return STTSM_ERR_CUDA;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)npiece};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)TC_KC, (cuuint32_t)box_rows, (cuuint32_t)npiece};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(xpieces), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? STTSM_OK : STTSM_ERR_CUDA;
}

}  // namespace sttsm

extern "C" {

int64_t bcss_num_blocks(int m, int64_t n, int b)
{
    if (m < 1 || m > 64 || n < 1 || b < 1) return -1;
    int64_t nbar = (n + b - 1) / b;
    double c = 1.0;
    for (int i = 1; i <= m; ++i) c = c * (double)(nbar - 1 + i) / i;
    if (c > 9.0e18) return -1;
    int64_t r = 1;
    for (int i = 1; i <= m; ++i) r = r * (nbar - 1 + i) / i;
    return r;
}

int64_t bcss_num_elems(int m, int64_t n, int b)
{
    int64_t nb = bcss_num_blocks(m, n, b);
    if (nb < 0) return -1;
    double e = (double)nb;
    int64_t r = nb;
    for (int a = 0; a < m; ++a) { e *= b; r *= b; }
    if (e > 9.0e18) return -1;
    return r;
}

int64_t bcss_block_rank(int m, const int32_t* s)
{
    if (m < 1 || m > STTSM_MAX_M || !s) return -1;
    for (int a = 0; a < m; ++a) {
        if (s[a] < 0 || (a > 0 && s[a] < s[a - 1])) return -1;
    }
    return colex_rank(s, m);
}

int bcss_block_unrank(int m, int64_t rank, int32_t* out)
{
    if (m < 1 || m > STTSM_MAX_M || rank < 0 || !out) return STTSM_ERR_ARG;
    colex_unrank(rank, m, out);
    return STTSM_OK;
}

double sttsm_flops(int m, int64_t n, int64_t p, int b)
{
    if (m < 1 || n < 1 || p < 1 || b < 1) return -1.0;
    const double nbar = (double)((n + b - 1) / b), pbar = (double)((p + b - 1) / b);
    auto C = [](double x, int y) {
        if (y < 0 || x < y) return 0.0;
        double c = 1.0;
        for (int i = 1; i <= y; ++i) c = c * (x - y + i) / i;
        return c;
    };
    double s = 0.0;
    for (int d = 0; d < m; ++d) s += C(pbar + d, d + 1) * C(nbar + m - d - 2, m - d - 1);
    double bp = 1.0;
    for (int a = 0; a <= m; ++a) bp *= b;
    return 2.0 * nbar * bp * s;
}

int bcss_pack(const void* dense, void* bcss, int m, int64_t n, int b, int dtype, void* stream)
{
    if (!dense || !bcss || m < 1 || m > STTSM_MAX_M || n < 1 || b < 1 || (dtype != 0 && dtype != 1)) return STTSM_ERR_ARG;
    if (bcss_num_elems(m, n, b) < 0 || bcss_num_blocks(m, n, b) >= (int64_t)1 << 31) return STTSM_ERR_UNSUPPORTED;
    return cuda_err(launch_bcss_pack(dense, bcss, m, n, b, dtype, (cudaStream_t)stream));
}

int bcss_unpack(const void* bcss, void* dense, int m, int64_t n, int b, int dtype, void* stream)
{
    if (!dense || !bcss || m < 1 || m > STTSM_MAX_M || n < 1 || b < 1 || (dtype != 0 && dtype != 1)) return STTSM_ERR_ARG;
    if (bcss_num_elems(m, n, b) < 0) return STTSM_ERR_UNSUPPORTED;
    return cuda_err(launch_bcss_unpack(bcss, dense, m, n, b, dtype, (cudaStream_t)stream));
}

int sttsm_workspace_size(int m, int64_t n, int64_t p, int b, int prec, size_t* bytes)
{
    if (!bytes) return STTSM_ERR_ARG;
    if (prec == STTSM_TF32X3) return STTSM_ERR_UNSUPPORTED;
    if (!prec_valid(prec)) return STTSM_ERR_ARG;
    Shape s;
    int rc = make_shape(m, n, p, b, &s);
    if (rc != STTSM_OK) return rc;
    *bytes = ws_layout(s, prec).total;
    return STTSM_OK;
}

int sttsm_device_status(void) { return take_status(); }

int sttsm_selftest_wait_timeout(double limit_ms)
{
    if (!(limit_ms > 0.0) || limit_ms > 1000.0) return STTSM_ERR_ARG;
    int* st = status_dev();
    if (!st) return STTSM_ERR_CUDA;
    if (take_status() != 0) return STTSM_ERR_TIMEOUT;   // an earlier timeout is reported first
    if (launch_wait_probe(st, (unsigned long long)(limit_ms * 1e6), nullptr) != 0) return STTSM_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return STTSM_ERR_CUDA;
    return take_status() != 0 ? STTSM_ERR_TIMEOUT : STTSM_OK;
}

int sttsm_set_small_kernel(int kind)
{
    if (kind != 0 && kind != 1) return STTSM_ERR_ARG;
    g_small_kind.store(kind);
    return STTSM_OK;
}

int sttsm_set_fused_tail(int mode)
{
    if (mode < 0 || mode > 2) return STTSM_ERR_ARG;
    g_fused_tail.store(mode);
    return STTSM_OK;
}

int sttsm_set_inblock_symmetry(int on)
{
    if (on != 0 && on != 1) return STTSM_ERR_ARG;
    g_inblock_sym.store(on);
    return STTSM_OK;
}

int sttsm_plan_sym_rows(int m, int64_t n, int64_t p, int b, int d, int64_t parent, int64_t rho0, int64_t count,
                        int64_t* g_out, uint32_t* tie_out, int64_t* rows_out)
{
    Shape s;
    int rc = make_shape(m, n, p, b, &s);
    if (rc != STTSM_OK) return rc;
    if (!sym_shape_ok(s)) return STTSM_ERR_UNSUPPORTED;
    if (d < 0 || d >= m || parent < 0 || parent >= s.lv[d].nodes_parent || rho0 < 0 || count < 0) return STTSM_ERR_ARG;
    SymTab T;
    sym_tab_fill(T, 0, 1);
    uint32_t pattern = 0;
    if (d > 0) {
        int32_t u[STTSM_MAX_M];
        colex_unrank(parent, d, u);
        for (int t = 0; t + 1 < d; ++t)
            if (u[t] == u[t + 1]) pattern |= 1u << t;
    }
    const int k = s.lv[d].k, Kp = (int)(s.nbar * b);
    const int64_t rows = sym_parent_rows(T, m, k, b, Kp, pattern);
    if (rows_out) *rows_out = rows;
    int32_t bpow[STTSM_MAX_M + 1];
    int64_t bp = 1;
    for (int a = 0; a <= STTSM_MAX_M; ++a) { bpow[a] = (int32_t)(bp < ((int64_t)1 << 31) ? bp : 0); bp *= b; }
    for (int64_t i = 0; i < count; ++i) {
        uint32_t tie = 0;
        const int64_t rho = rho0 + i;
        uint32_t iblk = 0;
        const int64_t g = rho < rows ? sym_row(T, m, k, b, Kp, s.R, bpow, pattern, rho, &tie, &iblk) : -1;
        if (g_out) g_out[i] = g;
        if (tie_out) tie_out[i] = tie;
    }
    return STTSM_OK;
}

int sttsm_profile_enable(int on)
{
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (on) prof_clear_locked();
    g_prof_on = on != 0;
    return STTSM_OK;
}

int sttsm_profile_read(int max, int* kind, int* level, double* flops, float* ms, int* count)
{
    std::lock_guard<std::mutex> lock(g_prof_mu);
    if (count) *count = (int)g_prof.size();
    for (int i = 0; i < (int)g_prof.size() && i < max; ++i) {
        ProfRec& r = g_prof[i];
        if (cudaEventSynchronize(r.b) != cudaSuccess) return STTSM_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return STTSM_ERR_CUDA;
        if (kind) kind[i] = r.kind;
        if (level) level[i] = r.level;
        if (flops) flops[i] = r.flops;
        if (ms) ms[i] = t;
    }
    return STTSM_OK;
}

int sttsm_plan_level(int m, int64_t n, int64_t p, int b, int prec, int d, int32_t* tiles, int64_t tiles_cap,
                     int32_t* G, int64_t G_cap, int64_t* ntiles_out, int64_t* nG_out, int64_t* info)
{
    if (prec == STTSM_TF32X3) return STTSM_ERR_UNSUPPORTED;
    if (!prec_valid(prec)) return STTSM_ERR_ARG;
    Shape s;
    int rc = make_shape(m, n, p, b, &s);
    if (rc != STTSM_OK) return rc;
    if (d < 0 || d >= m) return STTSM_ERR_ARG;
    const bool fp64 = prec == STTSM_FP64;
    int BM = fp64 ? 64 : TC_BM, BN = fp64 ? 64 : (tc_small_mode(s) ? TC_SMALL_BN : TC_BN);
    const bool gathered = !fp64 && !tc_small_mode(s) && !tc_tma_mode(s);
    if (prec_r64(prec) && (d == m - 1 || gathered) && BN > R64_BN) BN = R64_BN;
    std::vector<Tile> tl;
    std::vector<int32_t> g;
    if (!fp64 && sym_levels(s, prec))
        build_level_tiles_sym(s, d, BM, BN, 0, tl);
    else
        build_level_tiles(s, d, BM, BN, 0, tl, !fp64 && tma_order16x8(s, d));
    build_level_G(s, d, g);
    if (ntiles_out) *ntiles_out = (int64_t)tl.size();
    if (nG_out) *nG_out = (int64_t)g.size();
    const LevelShape& L = s.lv[d];
    if (info) {
        int64_t v[9] = {L.k, L.P_parent, L.P_out, L.P_out * s.R, L.nodes_parent, L.nodes_out, s.R, s.bm, BM};
        for (int i = 0; i < 9; ++i) info[i] = v[i];
    }
    if (tiles) {
        if (tiles_cap < (int64_t)tl.size()) return STTSM_ERR_NOMEM;
        memcpy(tiles, tl.data(), tl.size() * sizeof(Tile));
    }
    if (G) {
        if (G_cap < (int64_t)g.size()) return STTSM_ERR_NOMEM;
        memcpy(G, g.data(), g.size() * sizeof(int32_t));
    }
    return STTSM_OK;
}

int sttsm_plan_pair(int m, int64_t n, int64_t p, int b, int32_t* tiles, int64_t tiles_cap, int64_t* ntiles_out,
                    int32_t* group_out)
{
    Shape s;
    int rc = make_shape(m, n, p, b, &s);
    if (rc != STTSM_OK) return rc;
    if (!pair_mode(s)) return STTSM_ERR_UNSUPPORTED;
    std::vector<Tile> tl;
    build_pair_tiles(s, 0, tl);
    if (ntiles_out) *ntiles_out = (int64_t)tl.size();
    if (group_out) *group_out = pair_group(s);
    if (tiles) {
        if (tiles_cap < (int64_t)tl.size()) return STTSM_ERR_NOMEM;
        memcpy(tiles, tl.data(), tl.size() * sizeof(Tile));
    }
    return STTSM_OK;
}

}  // extern "C"

namespace sttsm {
namespace {

// Levels 0 .. nlev-1 of the chain (nlev = m: C; nlev = m - 1: the all-but-one
// result T^(1)); the last of them writes `C` (FP32 / FP64), the others the
// workspace's ping-pong buffers.
int run_chain(const void* A, const void* X, int m, int64_t n, int64_t p, int b, void* C, int prec,
              void* workspace, size_t ws_bytes, void* stream_, int nlev)
{
    if (!A || !X || !C) return STTSM_ERR_ARG;
    if (prec == STTSM_TF32X3) return STTSM_ERR_UNSUPPORTED;
    if (!prec_valid(prec)) return STTSM_ERR_ARG;
    if (!aligned(A, 16) || !aligned(X, 16) || !aligned(C, 16)) return STTSM_ERR_ARG;
    if (n >= (int64_t)1 << 30 || p >= (int64_t)1 << 30) return STTSM_ERR_UNSUPPORTED;
    Shape s;
    int rc = make_shape(m, n, p, b, &s);
    if (rc != STTSM_OK) return rc;
    const WsLayout w = ws_layout(s, prec);
    if (w.total > 0 && (!workspace || ws_bytes < w.total || !aligned(workspace, 256))) return STTSM_ERR_NOMEM;
    int* st = status_dev();
    if (!st) return STTSM_ERR_CUDA;
    if (take_status() != 0) return STTSM_ERR_TIMEOUT;
    cudaStream_t stream = (cudaStream_t)stream_;
    const bool fp64 = prec == STTSM_FP64;
    const bool small = !fp64 && tc_small_mode(s);
    const bool r64 = prec_r64(prec);
    // R64: the gathered kernel sums in FP64 at every level (as in batches and serving),
    // the TMA kernel at the last level; both then take tiles of at most 128 columns
    const bool gathered = !fp64 && !small && !tc_tma_mode(s);
    const int BM = fp64 ? 64 : TC_BM;
    const int BN = fp64 ? 64 : small ? TC_SMALL_BN : (r64 && gathered) ? R64_BN : TC_BN;
    // in-block symmetry: canonical entries only (short contractions, FP32 kernel)
    const bool sym = !fp64 && sym_levels(s, prec);
    const DevPlan* P = get_dev_plan(m, n, p, b, BM, BN, r64 && BN > R64_BN ? R64_BN : BN, sym);
    if (!P) return STTSM_ERR_NOMEM;
    char* ws = (char*)workspace;
    void* bufs[2] = {ws + w.buf0, ws + w.buf1};
    const int sms = num_sms();
    const int np = npiece_of(prec);
    if (w.tma) {
        // TMA-fed kernel: split X and A once, temporaries as BF16 pieces
        TmaInst tm;
        memset(&tm, 0, sizeof(tm));
        {
            ProfScope ps(stream, 2, -1, 0.0);
            rc = cuda_err(launch_split_x((const float*)X, ws + w.xpieces, (int)p, (int)n, w.rows, w.Kp, np, stream));
            if (rc == STTSM_OK)
                rc = cuda_err(launch_split_bcss((const float*)A, ws + w.apieces, s.lv[0].P_parent, s.bm, np, stream));
        }
        if (rc != STTSM_OK) return rc;
        for (int xs = 0; xs < TMA_NX && rc == STTSM_OK; ++xs)
            rc = make_x_tensor_map(&tm.tmX[xs], ws + w.xpieces, np, w.rows, w.Kp, 32 * (xs + 1));
        if (rc != STTSM_OK) return rc;
        for (int d = 0; d < nlev; ++d) {
            const LevelShape& LS = s.lv[d];
            const void* parent = d == 0 ? (const void*)(ws + w.apieces) : bufs[(d - 1) & 1];
            const bool o16 = tma_order16x8(s, d);
            rc = make_a_tensor_maps(tm.tmA, parent, LS.nodes_parent * LS.P_parent, np, b, m, LS.k, o16);
            if (rc != STTSM_OK) return rc;
            LevelInst& L = tm.L;
            L.parent = parent;
            L.out = d == nlev - 1 ? C : bufs[d & 1];
            L.out_np = d == nlev - 1 ? 0 : np;
            L.G = P->d_G[d];
            L.OFF = P->d_G[d] + level_G_size(s, d);
            L.X = X;
            L.m = m; L.b = b; L.k = LS.k; L.nbar = (int32_t)s.nbar;
            L.n = (int32_t)n; L.p = (int32_t)p;
            L.R = (int32_t)s.R;
            L.Ktot = (int32_t)(s.nbar * b);
            L.bm = s.bm;
            L.P_parent = LS.P_parent;
            L.P_out = LS.P_out;
            L.rows_per_parent = LS.P_out * s.R;
            L.order16x8 = o16 ? 1 : 0;
            int64_t bp = 1;
            for (int a = 0; a <= STTSM_MAX_M; ++a) { L.bpow[a] = (int32_t)(bp < ((int64_t)1 << 31) ? bp : 0); bp *= b; }
            const double lflops = (double)LS.nodes_out * (double)LS.P_out * (double)s.nbar * 2.0 * (double)s.bm * b;
            ProfScope ps(stream, 3, d, lflops);
            const int out_kind = d < nlev - 1 ? TMA_OUT_PIECES
                                 : d == m - 1 ? (r64 ? TMA_OUT_C64 : TMA_OUT_C) : TMA_OUT_F32;
            rc = cuda_err(launch_level_tma(np, tm, nullptr, P->d_tiles[d], P->ntiles[d], sms, st, out_kind, tma_sw32(s),
                                           P->maxcols[d], stream));
            if (rc != STTSM_OK) return rc;
        }
        return STTSM_OK;
    }
    TcInst ti;
    memset(&ti, 0, sizeof(ti));
    if (!fp64) {
        {
            ProfScope ps(stream, 2, -1, 0.0);
            rc = cuda_err(launch_split_x((const float*)X, ws + w.xpieces, (int)p, (int)n, w.rows, w.Kp, np, stream));
        }
        if (rc != STTSM_OK) return rc;
        rc = make_x_tensor_map(&ti.tmX, ws + w.xpieces, np, w.rows, w.Kp, small ? TC_SMALL_BN : TC_BN);
        if (rc != STTSM_OK) return rc;
    }
    // short contractions in FP32: the last two levels in one launch, T^(1) in shared memory
    const bool pair = small && small_kernel_kind() == 0 && fused_tail_enabled() && nlev == m && P->d_pair && !r64 && !sym;
    for (int d = 0; d < nlev; ++d) {
        const LevelShape& LS = s.lv[d];
        LevelInst& L = ti.L;
        const bool fused = pair && d == m - 2;
        L.parent = d == 0 ? A : bufs[(d - 1) & 1];
        L.out = (d == nlev - 1 || fused) ? C : bufs[d & 1];
        L.sym_full = d == nlev - 1 ? 1 : 0;
        L.G = P->d_G[d];
        L.OFF = P->d_G[d] + level_G_size(s, d);
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
        double lflops = (double)LS.nodes_out * (double)LS.P_out * (double)s.nbar * 2.0 * (double)s.bm * b;
        if (fused) {
            const LevelShape& L2 = s.lv[m - 1];
            lflops += (double)L2.nodes_out * (double)L2.P_out * (double)s.nbar * 2.0 * (double)s.bm * b;
            ProfScope ps(stream, 4, d, lflops);
            rc = cuda_err(launch_level_pair_f32(L, nullptr, P->d_pair, P->npair, sms, stream));
            if (rc != STTSM_OK) return rc;
            break;   // level m-1 is done too
        }
        ProfScope ps(stream, fp64 ? 0 : 1, d, lflops);
        if (fp64) rc = cuda_err(launch_level_fp64(L, nullptr, P->d_tiles[d], P->ntiles[d], sms, stream));
        // the R64 precisions: the last level sums in FP64 (the FP32 kernel for short contractions)
        else if (small && (small_kernel_kind() == 0 || r64))
            rc = cuda_err(launch_level_small_f32(L, nullptr, P->d_tiles[d], P->ntiles[d], sms, stream, r64 && d == m - 1,
                                                 sym ? 1 : 0));
        else if (small) rc = cuda_err(launch_level_tc_small(np, ti, nullptr, P->d_tiles[d], P->ntiles[d], sms, st, stream));
        else if (r64)
            rc = cuda_err(launch_level_tc_r64(np, ti, nullptr, P->d_tiles[d], P->ntiles[d], sms, st, P->maxcols[d], stream));
        else rc = cuda_err(launch_level_tc(np, ti, nullptr, P->d_tiles[d], P->ntiles[d], sms, st, stream));
        if (rc != STTSM_OK) return rc;
    }
    return STTSM_OK;
}

}  // namespace
}  // namespace sttsm

extern "C" {

int sttsm_bcss(const void* A, const void* X, int m, int64_t n, int64_t p, int b, void* C, int prec,
               void* workspace, size_t ws_bytes, void* stream)
{
    return sttsm::run_chain(A, X, m, n, p, b, C, prec, workspace, ws_bytes, stream, m);
}

int sttsm_bcss_all_but_one(const void* A, const void* X, int m, int64_t n, int64_t p, int b, void* T, int prec,
                           void* workspace, size_t ws_bytes, void* stream)
{
    if (m < 2) return STTSM_ERR_ARG;
    return sttsm::run_chain(A, X, m, n, p, b, T, prec, workspace, ws_bytes, stream, m - 1);
}

int64_t sttsm_all_but_one_elems(int m, int64_t n, int64_t p, int b)
{
    if (m < 2 || m > STTSM_MAX_M || n < 1 || p < 1 || b < 1) return -1;
    const int64_t nbar = (n + b - 1) / b, pbar = (p + b - 1) / b;
    // C(pbar + m - 2, m - 1) sorted (m-1)-tuples of p-blocks, nbar blocks each
    double c = 1.0;
    for (int i = 1; i <= m - 1; ++i) c = c * (double)(pbar - 1 + i) / i;
    double e = c * (double)nbar;
    for (int a = 0; a < m; ++a) e *= b;
    if (e > 9.0e18) return -1;
    int64_t r = 1;
    for (int i = 1; i <= m - 1; ++i) r = r * (pbar - 1 + i) / i;
    r *= nbar;
    for (int a = 0; a < m; ++a) r *= b;
    return r;
}

double sttsm_all_but_one_flops(int m, int64_t n, int64_t p, int b)
{
    if (m < 2 || n < 1 || p < 1 || b < 1) return -1.0;
    const double nbar = (double)((n + b - 1) / b), pbar = (double)((p + b - 1) / b);
    auto C = [](double x, int y) {
        if (y < 0 || x < y) return 0.0;
        double c = 1.0;
        for (int i = 1; i <= y; ++i) c = c * (x - y + i) / i;
        return c;
    };
    double s = 0.0;
    for (int d = 0; d < m - 1; ++d) s += C(pbar + d, d + 1) * C(nbar + m - d - 2, m - d - 1);
    double bp = 1.0;
    for (int a = 0; a <= m; ++a) bp *= b;
    return 2.0 * nbar * bp * s;
}

int sttsm_bcss_host(const void* A, const void* X, int m, int64_t n, int64_t p, int b, void* C, int prec,
                    void* dA, void* dX, void* dC, void* workspace, size_t ws_bytes, void* stream_)
{
    if (!A || !X || !C || !dA || !dX || !dC) return STTSM_ERR_ARG;
    const size_t esz = prec == STTSM_FP64 ? 8 : 4;
    const int64_t na = bcss_num_elems(m, n, b), nc = bcss_num_elems(m, p, b);
    if (na < 0 || nc < 0) return STTSM_ERR_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (cudaMemcpyAsync(dA, A, (size_t)na * esz, cudaMemcpyHostToDevice, stream) != cudaSuccess) return STTSM_ERR_CUDA;
    if (cudaMemcpyAsync(dX, X, (size_t)(p * n) * esz, cudaMemcpyHostToDevice, stream) != cudaSuccess) return STTSM_ERR_CUDA;
    int rc = sttsm_bcss(dA, dX, m, n, p, b, dC, prec, workspace, ws_bytes, stream_);
    if (rc != STTSM_OK) return rc;
    if (cudaMemcpyAsync(C, dC, (size_t)nc * esz, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return STTSM_ERR_CUDA;
    return STTSM_OK;
}

}  // extern "C"
