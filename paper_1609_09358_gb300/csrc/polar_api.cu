// polar_api.cu -- the C ABI of include/polar_gb300.h: argument checks, the per-device code-table
// cache, workspace layout and kernel dispatch.  Every decoding step runs in the kernels of
// bp_kernel.cuh, scl_kernel.cuh and encode_kernels.cuh; nothing here touches frame data.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "bp_launch.cuh"
#include "encode_kernels.cuh"
#include "polar_common.cuh"
#include "mixed_kernels.cuh"
#include "scl_kernel.cuh"
#include "wms_kernels.cuh"

namespace polar {

// ---------------------------------------------------------------------------- errors
static thread_local std::string g_last_error;

static int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

static int cuda_fail(cudaError_t e, const char* what)
{
    return fail(POLAR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define POLAR_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------- code tables
__device__ DevCode g_codes[POLAR_MAX_CODES];

struct DeviceCodes {
    bool init = false;
    DevCode* base = nullptr;  // device address of g_codes on this device
    std::vector<DevCode> host;  // host copies of the filled slots, in slot order
};
static std::mutex g_codes_mutex;
static std::vector<DeviceCodes> g_dev;

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int log2i(int v)
{
    int n = 0;
    while ((1 << n) < v) ++n;
    return n;
}

static int check_code(const polar_code* code)
{
    if (!code) return fail(POLAR_ERR_ARG, "code is NULL");
    const int N = code->N, K = code->K, c = code->crc_len;
    if (!is_pow2(N) || N < POLAR_MIN_N || N > POLAR_MAX_N)
        return fail(POLAR_ERR_ARG, "N = %d: must be a power of two in [%d, %d]", N, POLAR_MIN_N, POLAR_MAX_N);
    if (!(c == 0 || c == 8 || c == 16 || c == 24)) return fail(POLAR_ERR_ARG, "crc_len = %d: must be 0, 8, 16 or 24", c);
    if (K < c || K > N) return fail(POLAR_ERR_ARG, "K = %d: must satisfy crc_len <= K <= N", K);
    if (c > 0 && (code->crc_poly >> c) != 0) return fail(POLAR_ERR_ARG, "crc_poly has bits above x^%d", c - 1);
    if (!code->frozen) return fail(POLAR_ERR_ARG, "frozen table is NULL");
    int info = 0;
    for (int i = 0; i < N; ++i) info += code->frozen[i] ? 0 : 1;
    if (info != K) return fail(POLAR_ERR_ARG, "frozen table has %d information positions, K = %d", info, K);
    if (code->scl_decided)
        for (int i = 0; i < N; ++i)
            if (code->scl_decided[i] && code->frozen[i])
                return fail(POLAR_ERR_ARG, "scl_decided marks the frozen position %d", i);
    return POLAR_OK;
}

// Derived tables of a code: information indices in ascending order, payload position of each
// node, and the syndrome column x^(K-1-k) mod g(x) of each information node.
static void derive_code(const polar_code* code, DevCode& d)
{
    memset(&d, 0, sizeof d);
    d.N = code->N;
    d.n = log2i(code->N);
    d.K = code->K;
    d.c = code->crc_len;
    d.P = code->K - code->crc_len;
    d.poly = code->crc_poly;
    std::vector<int> info;
    for (int i = 0; i < d.N; ++i) {
        d.paypos[i] = -1;
        if (code->frozen[i])
            d.frozen_bits[i >> 5] |= 1u << (i & 31);
        else
            info.push_back(i);
        if (code->scl_decided && code->scl_decided[i]) d.decided_bits[i >> 5] |= 1u << (i & 31);
    }
    // powers x^m mod g(x), m = 0..K-1, by repeated multiplication with x
    std::vector<uint32_t> pw(d.K > 0 ? d.K : 1);
    uint32_t r = 1;
    const uint32_t top = d.c > 0 ? (1u << d.c) : 0u;
    for (int m = 0; m < d.K; ++m) {
        pw[m] = d.c > 0 ? r : 0u;
        if (d.c > 0) {
            r <<= 1;
            if (r & top) r ^= top | d.poly;
        }
    }
    for (int k = 0; k < d.K; ++k) {
        const int j = info[k];
        d.info_idx[k] = (int16_t)j;
        d.colsyn[j] = pw[d.K - 1 - k];
        if (k < d.P) d.paypos[j] = (int16_t)k;
    }
}

// Device pointer of the table slot holding `code` on the current device; fills a free slot on
// first use (an asynchronous copy on `stream`).
static int code_slot(const polar_code* code, cudaStream_t stream, const DevCode** out)
{
    int rc = check_code(code);
    if (rc) return rc;
    DevCode d;
    derive_code(code, d);
    int dev = 0;
    POLAR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_codes_mutex);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DeviceCodes& dc = g_dev[dev];
    if (!dc.init) {
        dc.host.reserve(POLAR_MAX_CODES);
        void* p = nullptr;
        POLAR_CUDA(cudaGetSymbolAddress(&p, g_codes));
        dc.base = static_cast<DevCode*>(p);
        dc.init = true;
    }
    for (size_t s = 0; s < dc.host.size(); ++s) {
        if (memcmp(&dc.host[s], &d, sizeof d) == 0) {
            *out = dc.base + s;
            return POLAR_OK;
        }
    }
    if ((int)dc.host.size() >= POLAR_MAX_CODES)
        return fail(POLAR_ERR_CAPACITY, "more than %d distinct codes used on device %d", POLAR_MAX_CODES, dev);
    dc.host.push_back(d);
    const size_t s = dc.host.size() - 1;
    cudaError_t e = cudaMemcpyAsync(dc.base + s, &dc.host[s], sizeof(DevCode), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        dc.host.pop_back();
        return cuda_fail(e, "upload of a code table");
    }
    *out = dc.base + s;
    return POLAR_OK;
}

// ---------------------------------------------------------------------------- workspace
// [header 256 B: fail count, SCL work counter, status word][fail list: int32 x B][SCL scratch]
struct WsHeader {
    int fail_count;
    int scl_next;
    int err;
};
constexpr size_t kHeaderBytes = 256;

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static size_t ws_bytes(const polar_code* code, int B, int L, int op);

// hybrid_decode: one BP launch over the batch, then one persistent CA-SCL launch over the
// frames it compacted.  (Cutting the batch into chunks whose CA-SCL overlaps later BP chunks was
// measured slower: each CA-SCL launch costs at least one frame's decoding latency, and the frames
// BP fails are the ones that run all i_max iterations, i.e. the last to leave BP.)
struct ChunkHdr {
    int fail_count;
    int scl_next;
    int bp_next;
    int pad;
};
static size_t hybrid_chunk_header_bytes(int) { return 256; }

// Device buffers of hybrid_decode_host: the whole batch's LLRs, bits, status and iterations, the
// BP work counters of the chunks, and the hybrid workspace of the batch.
struct HostSet {
    size_t llr, bits, status, iters, counters, ws, ws_bytes, total;
};
// Chunk c of hybrid_decode_host: sizes 4096, 8192, then POLAR_HOST_CHUNK frames (small first
// chunks so that BP starts early), the last one ragged.
static int host_chunk_size(int c) { return std::min(POLAR_HOST_CHUNK, 4096 << std::min(c, 8)); }
static int host_chunks(int B)
{
    int c = 0;
    for (int b0 = 0; b0 < B; ++c) b0 += host_chunk_size(c);
    return std::max(1, c);
}
static HostSet host_set_layout(const polar_code* code, int B, int L)
{
    HostSet h{};
    const size_t row = (size_t)(code->K - code->crc_len + 7) / 8;
    size_t o = 0;
    h.llr = o;
    o = align_up(o + (size_t)B * code->N * sizeof(float), 256);
    h.bits = o;
    o = align_up(o + (size_t)B * row, 256);
    h.status = o;
    o = align_up(o + (size_t)B, 256);
    h.iters = o;
    o = align_up(o + (size_t)B * sizeof(uint16_t), 256);
    h.counters = o;
    o = align_up(o + sizeof(int) * (size_t)host_chunks(B), 256);
    h.ws = o;
    h.ws_bytes = ws_bytes(code, B, L, POLAR_OP_HYBRID);
    o = align_up(o + h.ws_bytes, 256);
    h.total = o;
    return h;
}

// Per-chunk counters of hybrid_decode_scheduled (chunks of at least kSchedMinChunk frames).
struct SchedHdr {
    int fail_count;
    int scl_next;
    int pad[2];
};
constexpr int kSchedMinChunk = 256;
static size_t sched_hdr_bytes(int B)
{
    return align_up(sizeof(SchedHdr) * (size_t)((std::max(B, 1) + kSchedMinChunk - 1) / kSchedMinChunk), 256);
}

static size_t ws_bytes(const polar_code* code, int B, int L, int op)
{
    if (op == POLAR_OP_BP) return 0;
    if (op == POLAR_OP_HYBRID_HOST) return host_set_layout(code, std::max(B, 1), L).total;
    size_t b = kHeaderBytes;
    if (op == POLAR_OP_HYBRID) {
        b += hybrid_chunk_header_bytes(B);
        b += align_up(sizeof(int) * (size_t)std::max(B, 1), 256);
    } else if (op == POLAR_OP_HYBRID_SCHED) {
        b += sched_hdr_bytes(B);
        b += align_up(sizeof(int) * (size_t)std::max(B, 1), 256);
    }
    b += scl_scratch_bytes(code->N, L);
    return b;
}

// library-owned streams per device: hybrid_decode_host's second compute stream [0] and copy stream
// [1]; hybrid_decode_scheduled's BP streams [2 .. 2 + POLAR_SCHED_BP_STREAMS) and CA-SCL stream
constexpr int kAuxStreams = 3 + POLAR_SCHED_BP_STREAMS;
static std::mutex g_aux_mutex;
static std::vector<cudaStream_t> g_aux;
static int aux_stream(int which, cudaStream_t* out)
{
    int dev = 0;
    POLAR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_aux_mutex);
    if ((int)g_aux.size() <= kAuxStreams * dev + which) g_aux.resize(kAuxStreams * (dev + 1), nullptr);
    cudaStream_t& sref = g_aux[kAuxStreams * dev + which];
    if (!sref) POLAR_CUDA(cudaStreamCreateWithFlags(&sref, cudaStreamNonBlocking));
    *out = sref;
    return POLAR_OK;
}



// ---------------------------------------------------------------------------- kernel timing
struct ProfRecord {
    int kind;  // 0 BP, 1 SCL
    cudaEvent_t start, stop;
};
struct ProfState {
    bool on = false;
    cudaError_t err = cudaSuccess;  // first failed event creation or record since the last read
    std::vector<ProfRecord> recs;
    std::vector<cudaEvent_t> pool;
};
static thread_local ProfState g_prof;

// An event from the pool or a new one; null (and the error kept for polar_profile_read) if it
// cannot be created, in which case the launch goes untimed.
static cudaEvent_t prof_event()
{
    if (!g_prof.pool.empty()) {
        cudaEvent_t e = g_prof.pool.back();
        g_prof.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    const cudaError_t rc = cudaEventCreate(&e);
    if (rc != cudaSuccess) {
        if (g_prof.err == cudaSuccess) g_prof.err = rc;
        return nullptr;
    }
    return e;
}

// Brackets one kernel launch with events when timing is enabled.
struct ProfScope {
    int kind;
    cudaStream_t st;
    cudaEvent_t start = nullptr;
    ProfScope(int k, cudaStream_t s) : kind(k), st(s)
    {
        if (g_prof.on && (start = prof_event()) != nullptr) {
            const cudaError_t rc = cudaEventRecord(start, st);
            if (rc != cudaSuccess) {
                if (g_prof.err == cudaSuccess) g_prof.err = rc;
                g_prof.pool.push_back(start);
                start = nullptr;
            }
        }
    }
    ~ProfScope()
    {
        if (!start) return;
        cudaEvent_t stop = prof_event();
        const cudaError_t rc = stop ? cudaEventRecord(stop, st) : cudaErrorUnknown;
        if (rc == cudaSuccess) {
            g_prof.recs.push_back({kind, start, stop});
        } else {
            if (stop && g_prof.err == cudaSuccess) g_prof.err = rc;
            g_prof.pool.push_back(start);
            if (stop) g_prof.pool.push_back(stop);
        }
    }
};

// BP variant bits carried in `precision` (bit 0 exact g, bit 1 re-encoding stop) and the message type
static int bp_variant(int precision)
{
    return ((precision & POLAR_G_EXACT) ? 1 : 0) | ((precision & POLAR_STOP_REENCODE) ? 2 : 0);
}
static int bp_message(int precision) { return precision & ~(POLAR_G_EXACT | POLAR_STOP_REENCODE | POLAR_WMS_UNIT); }

static int launch_bp(const DevCode* dcode, const polar_code* code, const float* llr, int B, int max_iters,
                     float llr_max, int precision, const void* w, int w_iters, uint8_t* bits, uint8_t* status,
                     uint16_t* iters, float* llr_u, float* llr_x, int* fail_count, int* fail_list,
                     cudaStream_t stream, int* fail_total = nullptr, int* next = nullptr, int fixed_iters = 0,
                     int frame0 = 0)
{
    BPArgs a{};
    a.frame0 = frame0;
    a.fixed_iters = fixed_iters;
    a.fail_total = fail_total;
    a.next = next;
    a.llr = llr;
    a.B = B;
    a.max_iters = max_iters;
    a.llr_max = llr_max;
    a.w = w;
    a.w_iters = w ? w_iters : 0;
    a.bits = bits;
    a.status = status;
    a.iters = iters;
    a.llr_u = llr_u;
    a.llr_x = llr_x;
    a.code = dcode;
    a.fail_count = fail_count;
    a.fail_list = fail_list;
    a.row_bytes = (code->K - code->crc_len + 7) / 8;
    const int n = log2i(code->N);
    if (B == 0) return POLAR_OK;
    if (n < 7 || n > 12) return fail(POLAR_ERR_ARG, "unsupported N = %d", code->N);
    if (w && code->N > POLAR_MAX_N_MIXED)
        return fail(POLAR_ERR_ARG, "learned weights: N = %d > %d", code->N, POLAR_MAX_N_MIXED);
    const int var = bp_variant(precision);
    const bool unit = (precision & POLAR_WMS_UNIT) != 0;
    precision = bp_message(precision);
    // learned scales: the half2 form with both frames of a register on the same iteration when
    // the caller vouches for scales within [-1, 1] and every iteration is a learned one
    const int weighted = !w ? 0 : (unit && precision == POLAR_FP16 && max_iters <= w_iters) ? 2 : 1;
    const BPKernelInfo k = precision == POLAR_FP16 ? bp_kernel_info_fp16(n, weighted, code->crc_len <= 16)
                           : var               ? bp_kernel_info_fp32_var(n, var)
                                               : bp_kernel_info_fp32(n, weighted, code->crc_len <= 16);
    if (!k.fn) return fail(POLAR_ERR_ARG, "no BP kernel for N = %d with these options", code->N);
    if (k.smem > 48 * 1024) {
        // above the default dynamic shared-memory limit (N = 4096); set once per kernel and device
        static std::mutex m;
        static std::vector<std::pair<int, const void*>> done;
        int dev = 0;
        POLAR_CUDA(cudaGetDevice(&dev));
        std::lock_guard<std::mutex> lock(m);
        if (std::find(done.begin(), done.end(), std::make_pair(dev, k.fn)) == done.end()) {
            POLAR_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
            done.push_back(std::make_pair(dev, k.fn));
        }
    }
    const int fpt = precision == POLAR_FP16 ? 2 : 1;
    const int groups = (B + fpt - 1) / fpt;
    const int F = k.groups_per_cta;
    int grid = (groups + F - 1) / F;
    if (next) {
        // persistent: as many CTAs as are resident at once; groups refill from the counter
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, k.threads, k.smem);
        if (e != cudaSuccess) return cuda_fail(e, "bp occupancy");
        grid = std::min(grid, std::max(1, per_sm) * scl_sm_count());
    }
    ProfScope prof(0, stream);
    void* args[] = {&a};
    const cudaError_t e = cudaLaunchKernel(k.fn, dim3(grid), dim3(k.threads), args, k.smem, stream);
    return e == cudaSuccess ? POLAR_OK : cuda_fail(e, "bp_kernel launch");
}

static int check_bp_args(const polar_code* code, const float* llr, int B, int max_iters, float llr_max,
                         int precision, const void* w, int w_iters, const uint8_t* bits, const uint8_t* status,
                         const uint16_t* iters)
{
    const int rc = check_code(code);
    if (rc) return rc;
    if (bp_variant(precision) && (bp_message(precision) != POLAR_FP32 || w))
        return fail(POLAR_ERR_ARG, "POLAR_G_EXACT / POLAR_STOP_REENCODE need POLAR_FP32 messages and no learned weights");
    precision = bp_message(precision);
    if (B < 0) return fail(POLAR_ERR_ARG, "B = %d < 0", B);
    if (max_iters < 1 || max_iters > 65535) return fail(POLAR_ERR_ARG, "max_iters = %d: must be in [1, 65535]", max_iters);
    if (!(llr_max > 0.0f) || !std::isfinite(llr_max)) return fail(POLAR_ERR_ARG, "llr_max must be finite and > 0");
    if (precision != POLAR_FP32 && precision != POLAR_FP16) return fail(POLAR_ERR_ARG, "precision = %d", precision);
    if (precision == POLAR_FP16 && llr_max > 32768.0f) return fail(POLAR_ERR_ARG, "llr_max > 32768 with FP16 messages");
    if (w && w_iters < 1) return fail(POLAR_ERR_ARG, "wms_iters = %d with weights given", w_iters);
    if (w && (reinterpret_cast<uintptr_t>(w) & 15u)) return fail(POLAR_ERR_ARG, "prepared weights not 16-byte aligned");
    if (B > 0 && (!llr || !status || !iters)) return fail(POLAR_ERR_ARG, "NULL llr/status/iters");
    if (B > 0 && !bits && code->K > code->crc_len) return fail(POLAR_ERR_ARG, "NULL bits");
    return POLAR_OK;
}

static const int kListSizes[] = {1, 2, 4, 8, 16, 32};
static bool valid_L(int L)
{
    for (int v : kListSizes)
        if (v == L) return true;
    return false;
}

static int launch_scl(const DevCode* dcode, const polar_code* code, const float* llr, int B, int L,
                      uint8_t* bits, uint8_t* status, const int* list, const int* count, int* next,
                      void* scratch, cudaStream_t stream)
{
    SCLArgs a{};
    a.llr = llr;
    a.B = B;
    a.L = L;
    a.bits = bits;
    a.status = status;
    a.code = dcode;
    a.list = list;
    a.count = count;
    a.next = next;
    a.scratch = static_cast<float*>(scratch);
    a.row_bytes = (code->K - code->crc_len + 7) / 8;
    ProfScope prof(1, stream);
    const cudaError_t e = scl_launch(a, code->N, L, stream);
    return e == cudaSuccess ? POLAR_OK : cuda_fail(e, "scl_kernel launch");
}

// ln Z of every bit-channel, one combining level at a time: each level splits every channel into
// its minus (index bit 0) and plus (index bit 1) child, so the first level decides the index MSB.
// minus: ln(2Z - Z^2), plus: 2 ln Z.
static std::vector<double> bhattacharyya_lnz(int N, double design_ebn0_db, double design_rate)
{
    const int n = log2i(N);
    std::vector<double> lz(1, -design_rate * std::pow(10.0, design_ebn0_db / 10.0)), next;
    for (int level = 0; level < n; ++level) {
        next.resize(lz.size() * 2);
        for (size_t i = 0; i < lz.size(); ++i) {
            const double v = lz[i];
            double minus;
            if (v <= -M_LN2) {
                minus = v + std::log(2.0 - std::exp(v));
            } else {
                const double d = -std::expm1(v);  // 1 - Z, accurate near Z = 1
                minus = std::log1p(-(d * d));
            }
            next[2 * i] = minus;
            next[2 * i + 1] = 2.0 * v;
        }
        lz.swap(next);
    }
    return lz;
}

// The PE functions of the BP kernels, elementwise: min-sum, exact (scalar form), exact (the packed
// pair form the FP32 kernels use; elements 2i and 2i+1 form a pair).  Unclipped.
__global__ void pe_eval_kernel(int op, const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out,
                               int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (op == POLAR_PE_EXACT_PACKED) {
        const int j = 2 * i;
        if (j >= n) return;
        const bool two = j + 1 < n;
        const float2 r = g_exact2(make_float2(a[j], two ? a[j + 1] : 0.0f), make_float2(b[j], two ? b[j + 1] : 0.0f));
        out[j] = r.x;
        if (two) out[j + 1] = r.y;
        return;
    }
    if (i >= n) return;
    out[i] = op == POLAR_PE_MINSUM ? xmin(a[i], b[i]) : g_exact(a[i], b[i]);
}

}  // namespace polar

using namespace polar;

// ==================================================================================== C ABI
extern "C" {

const char* polar_last_error(void) { return g_last_error.c_str(); }

int polar_reliability(int32_t N, double design_ebn0_db, double design_rate, double* lnz_out)
{
    if (!is_pow2(N) || N < 2 || N > (1 << 20)) return fail(POLAR_ERR_ARG, "N = %d: power of two in [2, 2^20]", N);
    if (!(design_rate > 0.0) || !std::isfinite(design_ebn0_db)) return fail(POLAR_ERR_ARG, "bad design point");
    if (!lnz_out) return fail(POLAR_ERR_ARG, "lnz_out is NULL");
    const std::vector<double> lz = bhattacharyya_lnz(N, design_ebn0_db, design_rate);
    for (int i = 0; i < N; ++i) lnz_out[i] = lz[i];
    return POLAR_OK;
}

int polar_construct(int32_t N, int32_t K, double design_ebn0_db, double design_rate, uint8_t* frozen_out,
                    int32_t* info_idx_out)
{
    if (!is_pow2(N) || N < 2 || N > (1 << 20)) return fail(POLAR_ERR_ARG, "N = %d: power of two in [2, 2^20]", N);
    if (K < 0 || K > N) return fail(POLAR_ERR_ARG, "K = %d outside [0, N]", K);
    if (!(design_rate > 0.0) || !std::isfinite(design_ebn0_db)) return fail(POLAR_ERR_ARG, "bad design point");
    if (!frozen_out) return fail(POLAR_ERR_ARG, "frozen_out is NULL");
    const std::vector<double> lz = bhattacharyya_lnz(N, design_ebn0_db, design_rate);
    std::vector<int> order(N);
    for (int i = 0; i < N; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (lz[a] != lz[b]) return lz[a] < lz[b];
        return a > b;  // equal reliability: the larger index counts as more reliable
    });
    for (int i = 0; i < N; ++i) frozen_out[i] = 1;
    for (int k = 0; k < K; ++k) frozen_out[order[k]] = 0;
    if (info_idx_out) {
        int k = 0;
        for (int i = 0; i < N; ++i)
            if (!frozen_out[i]) info_idx_out[k++] = i;
    }
    return POLAR_OK;
}

int polar_encode(const polar_code* code, const uint8_t* payload, int32_t B, uint8_t* codeword, void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (B < 0) return fail(POLAR_ERR_ARG, "B < 0");
    const DevCode* d = nullptr;
    int rc = code_slot(code, st, &d);
    if (rc) return rc;
    if (B == 0) return POLAR_OK;
    if (!codeword || (!payload && code->K > code->crc_len)) return fail(POLAR_ERR_ARG, "NULL payload/codeword");
    const int warps = 4;
    encode_kernel<<<(B + warps - 1) / warps, warps * 32, 0, st>>>(d, payload, B, (code->K - code->crc_len + 7) / 8,
                                                                codeword);
    POLAR_CUDA(cudaGetLastError());
    return POLAR_OK;
}

int polar_random_payload(int32_t B, int32_t P, uint64_t seed, uint64_t frame0, uint8_t* payload, void* stream)
{
    if (B < 0 || P < 0) return fail(POLAR_ERR_ARG, "B or P < 0");
    if (B == 0 || P == 0) return POLAR_OK;
    if (!payload) return fail(POLAR_ERR_ARG, "NULL payload");
    const long long total = (long long)B * (((P + 31) / 32 + 3) / 4);
    random_payload_kernel<<<(unsigned)((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        B, P, seed, frame0, payload);
    POLAR_CUDA(cudaGetLastError());
    return POLAR_OK;
}

int polar_awgn_llr(const uint8_t* codeword, int32_t B, int32_t N, float sigma, const float* sigma_per_frame,
                   uint64_t seed, uint64_t frame0, float* llr, void* stream)
{
    if (B < 0 || !is_pow2(N) || N < 8 || (!sigma_per_frame && !(sigma > 0.0f)))
        return fail(POLAR_ERR_ARG, "bad B, N or sigma");
    if (B == 0) return POLAR_OK;
    if (!codeword || !llr) return fail(POLAR_ERR_ARG, "NULL codeword/llr");
    const long long total = (long long)B * (N / 4);
    awgn_llr_kernel<<<(unsigned)((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        codeword, B, N, sigma, sigma_per_frame, seed, frame0, llr);
    POLAR_CUDA(cudaGetLastError());
    return POLAR_OK;
}

size_t polar_workspace_bytes(const polar_code* code, int32_t B, int32_t L, int32_t op)
{
    if (check_code(code) != POLAR_OK || B < 0) return 0;
    if (op != POLAR_OP_BP && !valid_L(L)) return 0;
    if (op < POLAR_OP_BP || op > POLAR_OP_HYBRID_SCHED) return 0;
    return ws_bytes(code, B, L, op);
}

int bp_decode(const polar_code* code, const float* llr, int32_t B, int32_t max_iters, float llr_max,
              int32_t precision, const void* wms_scales, int32_t wms_iters, uint8_t* bits, uint8_t* status,
              uint16_t* iters, float* llr_u, float* llr_x, void* workspace, size_t ws, void* stream)
{
    (void)workspace;
    (void)ws;
    const int fixed_iters = (precision & POLAR_FIXED_ITERS) != 0;
    precision &= ~POLAR_FIXED_ITERS;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_bp_args(code, llr, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status, iters);
    if (rc) return rc;
    const DevCode* d = nullptr;
    if ((rc = code_slot(code, st, &d))) return rc;
    return launch_bp(d, code, llr, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status, iters,
                     llr_u, llr_x, nullptr, nullptr, st, nullptr, nullptr, fixed_iters);
}

int scl_decode(const polar_code* code, const float* llr, int32_t B, int32_t L, uint8_t* bits, uint8_t* status,
               void* workspace, size_t ws, void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_code(code);
    if (rc) return rc;
    if (B < 0) return fail(POLAR_ERR_ARG, "B < 0");
    if (!valid_L(L)) return fail(POLAR_ERR_ARG, "L = %d: must be 1, 2, 4, 8, 16 or 32", L);
    const DevCode* d = nullptr;
    rc = code_slot(code, st, &d);
    if (rc) return rc;
    if (B == 0) return POLAR_OK;
    if (!llr || !status || (!bits && code->K > code->crc_len)) return fail(POLAR_ERR_ARG, "NULL llr/bits/status");
    const size_t need = ws_bytes(code, B, L, POLAR_OP_SCL);
    if (!workspace || ws < need) return fail(POLAR_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws, need);
    char* base = static_cast<char*>(workspace);
    WsHeader* h = reinterpret_cast<WsHeader*>(base);
    POLAR_CUDA(cudaMemsetAsync(h, 0, sizeof(WsHeader), st));
    return launch_scl(d, code, llr, B, L, bits, status, nullptr, nullptr, &h->scl_next, base + kHeaderBytes, st);
}

int hybrid_decode(const polar_code* code, const float* llr, int32_t B, int32_t max_iters, float llr_max,
                  int32_t precision, const void* wms_scales, int32_t wms_iters, int32_t L, uint8_t* bits,
                  uint8_t* status, uint16_t* iters, void* workspace, size_t ws, void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_bp_args(code, llr, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status, iters);
    if (rc) return rc;
    if (!valid_L(L)) return fail(POLAR_ERR_ARG, "L = %d: must be 1, 2, 4, 8, 16 or 32", L);
    const DevCode* d = nullptr;
    if ((rc = code_slot(code, st, &d))) return rc;
    if (B == 0) return POLAR_OK;
    const size_t need = ws_bytes(code, B, L, POLAR_OP_HYBRID);
    if (!workspace || ws < need) return fail(POLAR_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws, need);
    // [total fail count (256 B)][counters (256 B)][fail list][SCL scratch]
    char* base = static_cast<char*>(workspace);
    int* total = reinterpret_cast<int*>(base);
    ChunkHdr* hdr = reinterpret_cast<ChunkHdr*>(base + kHeaderBytes);
    int* list = reinterpret_cast<int*>(base + kHeaderBytes + hybrid_chunk_header_bytes(B));
    void* scratch = reinterpret_cast<char*>(list) + align_up(sizeof(int) * (size_t)B, 256);
    POLAR_CUDA(cudaMemsetAsync(base, 0, kHeaderBytes + sizeof(ChunkHdr), st));
    if ((rc = launch_bp(d, code, llr, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status, iters,
                        nullptr, nullptr, &hdr->fail_count, list, st, total, &hdr->bp_next)))
        return rc;
    return launch_scl(d, code, llr, B, L, bits, status, list, &hdr->fail_count, &hdr->scl_next, scratch, st);
}

int hybrid_decode_host(const polar_code* code, const float* llr_host, int32_t B, int32_t max_iters, float llr_max,
                       int32_t precision, const void* wms_scales, int32_t wms_iters, int32_t L, uint8_t* bits_host,
                       uint8_t* status_host, uint16_t* iters_host, void* workspace, size_t ws, void* stream)
{
    cudaStream_t st0 = static_cast<cudaStream_t>(stream);
    int rc = check_bp_args(code, llr_host, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits_host,
                           status_host, iters_host);
    if (rc) return rc;
    if (!valid_L(L)) return fail(POLAR_ERR_ARG, "L = %d: must be 1, 2, 4, 8, 16 or 32", L);
    const DevCode* d = nullptr;
    if ((rc = code_slot(code, st0, &d))) return rc;
    if (B == 0) return POLAR_OK;
    const size_t need = ws_bytes(code, B, L, POLAR_OP_HYBRID_HOST);
    if (!workspace || ws < need) return fail(POLAR_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws, need);
    cudaStream_t st1 = nullptr, stc = nullptr;
    if ((rc = aux_stream(0, &st1)) || (rc = aux_stream(1, &stc))) return rc;
    const HostSet hs = host_set_layout(code, B, L);
    const size_t N = (size_t)code->N, row = (size_t)(code->K - code->crc_len + 7) / 8;
    char* base = static_cast<char*>(workspace);
    float* llr_d = reinterpret_cast<float*>(base + hs.llr);
    uint8_t* bits_d = reinterpret_cast<uint8_t*>(base + hs.bits);
    uint8_t* status_d = reinterpret_cast<uint8_t*>(base + hs.status);
    uint16_t* iters_d = reinterpret_cast<uint16_t*>(base + hs.iters);
    int* counters = reinterpret_cast<int*>(base + hs.counters);
    char* wsb = base + hs.ws;
    int* total = reinterpret_cast<int*>(wsb);
    ChunkHdr* hdr = reinterpret_cast<ChunkHdr*>(wsb + kHeaderBytes);
    int* list = reinterpret_cast<int*>(wsb + kHeaderBytes + hybrid_chunk_header_bytes(B));
    void* scratch = reinterpret_cast<char*>(list) + align_up(sizeof(int) * (size_t)B, 256);
    const int nchunks = host_chunks(B);
    POLAR_CUDA(cudaMemsetAsync(wsb, 0, kHeaderBytes + sizeof(ChunkHdr), st0));
    POLAR_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * (size_t)nchunks, st0));
    std::vector<cudaEvent_t> evs;
    auto event = [&](cudaEvent_t* e) -> int {
        POLAR_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        evs.push_back(*e);
        return POLAR_OK;
    };
    // The copy stream runs ahead, chunk by chunk; each chunk's BP launch waits for its own copy only,
    // and the chunks alternate between two compute streams (one chunk's last frames overlap the next
    // chunk).  One CA-SCL launch then takes every frame BP failed, and one copy brings the results
    // back.
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if ((rc = event(&ev0))) return rc;
    POLAR_CUDA(cudaEventRecord(ev0, st0));
    POLAR_CUDA(cudaStreamWaitEvent(stc, ev0, 0));
    POLAR_CUDA(cudaStreamWaitEvent(st1, ev0, 0));
    const cudaStream_t sts[2] = {st0, st1};
    for (int c = 0, b0 = 0; c < nchunks && rc == POLAR_OK; b0 += host_chunk_size(c), ++c) {
        const int nb = std::min(host_chunk_size(c), B - b0);
        const cudaStream_t st = sts[c & 1];
        cudaEvent_t evc = nullptr;
        if ((rc = event(&evc))) break;
        POLAR_CUDA(cudaMemcpyAsync(llr_d + (size_t)b0 * N, llr_host + (size_t)b0 * N, (size_t)nb * N * sizeof(float),
                                   cudaMemcpyHostToDevice, stc));
        POLAR_CUDA(cudaEventRecord(evc, stc));
        POLAR_CUDA(cudaStreamWaitEvent(st, evc, 0));
        rc = launch_bp(d, code, llr_d, nb, max_iters, llr_max, precision, wms_scales, wms_iters, bits_d, status_d,
                       iters_d, nullptr, nullptr, &hdr->fail_count, list, st, total, counters + c, 0, b0);
    }
    if (rc == POLAR_OK && (rc = event(&ev1)) == POLAR_OK) {
        POLAR_CUDA(cudaEventRecord(ev1, st1));
        POLAR_CUDA(cudaStreamWaitEvent(st0, ev1, 0));
        rc = launch_scl(d, code, llr_d, B, L, bits_d, status_d, list, &hdr->fail_count, &hdr->scl_next, scratch, st0);
    }
    if (rc == POLAR_OK) {
        if (row) POLAR_CUDA(cudaMemcpyAsync(bits_host, bits_d, (size_t)B * row, cudaMemcpyDeviceToHost, st0));
        POLAR_CUDA(cudaMemcpyAsync(status_host, status_d, (size_t)B, cudaMemcpyDeviceToHost, st0));
        POLAR_CUDA(cudaMemcpyAsync(iters_host, iters_d, (size_t)B * sizeof(uint16_t), cudaMemcpyDeviceToHost, st0));
    }
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    return rc;
}

// page-locked host copies of the chunks' failure counts (hybrid_decode_scheduled; calls serialise)
static std::mutex g_sched_mutex;
static int* g_sched_counts = nullptr;
static size_t g_sched_cap = 0;

int hybrid_decode_scheduled(const polar_code* code, const float* llr, int32_t B, int32_t max_iters, float llr_max,
                            int32_t precision, const void* wms_scales, int32_t wms_iters, int32_t L, int32_t chunk,
                            uint8_t* bits, uint8_t* status, uint16_t* iters, void* workspace, size_t ws, void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_bp_args(code, llr, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status, iters);
    if (rc) return rc;
    if (!valid_L(L)) return fail(POLAR_ERR_ARG, "L = %d: must be 1, 2, 4, 8, 16 or 32", L);
    if (chunk < kSchedMinChunk) return fail(POLAR_ERR_ARG, "chunk = %d: must be >= %d", chunk, kSchedMinChunk);
    const DevCode* d = nullptr;
    if ((rc = code_slot(code, st, &d))) return rc;
    if (B == 0) return POLAR_OK;
    const size_t need = ws_bytes(code, B, L, POLAR_OP_HYBRID_SCHED);
    if (!workspace || ws < need) return fail(POLAR_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws, need);
    char* base = static_cast<char*>(workspace);
    SchedHdr* hdr = reinterpret_cast<SchedHdr*>(base + kHeaderBytes);
    int* list = reinterpret_cast<int*>(base + kHeaderBytes + sched_hdr_bytes(B));
    void* scratch = reinterpret_cast<char*>(list) + align_up(sizeof(int) * (size_t)B, 256);
    const int nchunks = (B + chunk - 1) / chunk;
    constexpr int S = POLAR_SCHED_BP_STREAMS;
    cudaStream_t sbp[S], sscl = nullptr;
    for (int i = 0; i < S; ++i)
        if ((rc = aux_stream(2 + i, &sbp[i]))) return rc;
    if ((rc = aux_stream(2 + S, &sscl))) return rc;

    std::lock_guard<std::mutex> lock(g_sched_mutex);
    if (g_sched_cap < (size_t)nchunks) {
        if (g_sched_counts) cudaFreeHost(g_sched_counts);
        g_sched_counts = nullptr;
        g_sched_cap = 0;
        POLAR_CUDA(cudaMallocHost(&g_sched_counts, sizeof(int) * (size_t)nchunks));
        g_sched_cap = (size_t)nchunks;
    }
    struct Events {
        std::vector<cudaEvent_t> v;
        ~Events()
        {
            for (cudaEvent_t e : v) cudaEventDestroy(e);
        }
    } evs;
    auto event = [&](cudaEvent_t* e) -> int {
        POLAR_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        evs.v.push_back(*e);
        return POLAR_OK;
    };
    cudaEvent_t ev0 = nullptr, ev_scl = nullptr, ev_bp[S];
    if ((rc = event(&ev0)) || (rc = event(&ev_scl))) return rc;
    for (int i = 0; i < S; ++i)
        if ((rc = event(&ev_bp[i]))) return rc;
    POLAR_CUDA(cudaMemsetAsync(hdr, 0, sizeof(SchedHdr) * (size_t)nchunks, st));
    POLAR_CUDA(cudaEventRecord(ev0, st));
    for (int i = 0; i < S; ++i) POLAR_CUDA(cudaStreamWaitEvent(sbp[i], ev0, 0));
    POLAR_CUDA(cudaStreamWaitEvent(sscl, ev0, 0));

    int slot[S];  // chunk in BP on each stream, -1 = free
    bool used[S];
    for (int i = 0; i < S; ++i) slot[i] = -1, used[i] = false;
    std::vector<int> waiting;  // chunks whose failed frames wait for CA-SCL
    bool scl_busy = false, scl_used = false;
    int next = 0, done = 0;
    using clock = std::chrono::steady_clock;
    auto last_progress = clock::now();
    while (rc == POLAR_OK && (done < nchunks || !waiting.empty())) {
        bool progress = false;
        // enough buffer space: start the next chunks' BP on free streams
        for (int i = 0; i < S && next < nchunks && rc == POLAR_OK; ++i) {
            if (slot[i] >= 0) continue;
            const int c = next++, b0 = c * chunk, nb = std::min(chunk, B - b0);
            rc = launch_bp(d, code, llr, nb, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status,
                           iters, nullptr, nullptr, &hdr[c].fail_count, list + b0, sbp[i], nullptr, nullptr, 0, b0);
            if (rc) break;
            POLAR_CUDA(cudaMemcpyAsync(&g_sched_counts[c], &hdr[c].fail_count, sizeof(int), cudaMemcpyDeviceToHost,
                                       sbp[i]));
            POLAR_CUDA(cudaEventRecord(ev_bp[i], sbp[i]));
            slot[i] = c;
            used[i] = progress = true;
        }
        if (rc) break;
        // BP finished: its chunk's failures (counted on the device) wait for CA-SCL
        for (int i = 0; i < S; ++i) {
            if (slot[i] < 0) continue;
            const cudaError_t e = cudaEventQuery(ev_bp[i]);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) return cuda_fail(e, "BP launch of a chunk");
            if (g_sched_counts[slot[i]] > 0) waiting.push_back(slot[i]);
            slot[i] = -1;
            ++done;
            progress = true;
        }
        // failures waiting and the CA-SCL stream idle: start CA-SCL on every waiting chunk
        if (!waiting.empty()) {
            if (scl_busy) {
                const cudaError_t e = cudaEventQuery(ev_scl);
                if (e != cudaSuccess && e != cudaErrorNotReady) return cuda_fail(e, "CA-SCL launch");
                scl_busy = e == cudaErrorNotReady;
            }
            if (!scl_busy) {
                for (int c : waiting) {
                    rc = launch_scl(d, code, llr, B, L, bits, status, list + (size_t)c * chunk, &hdr[c].fail_count,
                                    &hdr[c].scl_next, scratch, sscl);
                    if (rc) break;
                }
                waiting.clear();
                POLAR_CUDA(cudaEventRecord(ev_scl, sscl));
                scl_busy = scl_used = progress = true;
            }
        }
        if (progress) {
            last_progress = clock::now();
        } else {
            if (clock::now() - last_progress > std::chrono::seconds(600))
                return fail(POLAR_ERR_TIMEOUT, "hybrid_decode_scheduled: no launch finished in 600 s");
            std::this_thread::yield();
        }
    }
    if (rc) return rc;
    // later work on `stream` follows every launch of the call
    if (scl_used) POLAR_CUDA(cudaStreamWaitEvent(st, ev_scl, 0));
    for (int i = 0; i < S; ++i)
        if (used[i]) POLAR_CUDA(cudaStreamWaitEvent(st, ev_bp[i], 0));
    return POLAR_OK;
}

size_t wms_prepared_bytes(const polar_code* code, int32_t wms_iters, int32_t precision)
{
    if (check_code(code) != POLAR_OK || wms_iters < 1 || code->N > POLAR_MAX_N_MIXED) return 0;
    if (precision != POLAR_FP32 && precision != POLAR_FP16) return 0;
    const size_t elem = precision == POLAR_FP16 ? 2 : 4;
    return (size_t)wms_iters * 2 * log2i(code->N) * code->N * elem;
}

int wms_prepare(const polar_code* code, const float* w, int32_t wms_iters, int32_t precision, void* prepared,
                size_t bytes, void* stream)
{
    int rc = check_code(code);
    if (rc) return rc;
    if (wms_iters < 1) return fail(POLAR_ERR_ARG, "wms_iters = %d < 1", wms_iters);
    if (precision != POLAR_FP32 && precision != POLAR_FP16) return fail(POLAR_ERR_ARG, "precision = %d", precision);
    const int n = log2i(code->N);
    if (n < 7 || code->N > POLAR_MAX_N_MIXED) return fail(POLAR_ERR_ARG, "learned weights: N = %d > %d", code->N,
                                                          POLAR_MAX_N_MIXED);
    if (!w || !prepared) return fail(POLAR_ERR_ARG, "NULL weights or output");
    if (reinterpret_cast<uintptr_t>(prepared) & 15u) return fail(POLAR_ERR_ARG, "output not 16-byte aligned");
    const size_t need = wms_prepared_bytes(code, wms_iters, precision);
    if (bytes < need) return fail(POLAR_ERR_WORKSPACE, "prepared buffer %zu < %zu bytes", bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = precision == POLAR_FP16 ? wms_prepare_fp16(n, w, wms_iters, prepared, st)
                                                  : wms_prepare_fp32(n, w, wms_iters, prepared, st);
    return e == cudaSuccess ? POLAR_OK : cuda_fail(e, "wms_prepare launch");
}

size_t wms_workspace_bytes(const polar_code* code, int32_t B, int32_t T)
{
    if (check_code(code) != POLAR_OK || B < 0 || T < 1 || code->N > POLAR_MAX_N_MIXED) return 0;
    const size_t n = (size_t)log2i(code->N), N = (size_t)code->N;
    return (size_t)B * (2 * (size_t)T * n * N + 3 * (n + 2) * N) * sizeof(float);
}

static int wms_common(const polar_code* code, const float* llr, int B, int T, float llr_max, const float* w,
                      void* workspace, size_t ws, cudaStream_t st, WMSArgs& a)
{
    int rc = check_code(code);
    if (rc) return rc;
    if (code->N > POLAR_MAX_N_MIXED) return fail(POLAR_ERR_ARG, "training: N = %d > %d", code->N, POLAR_MAX_N_MIXED);
    if (B < 0 || T < 1 || T > 1000) return fail(POLAR_ERR_ARG, "B = %d, T = %d", B, T);
    if (!(llr_max > 0.0f)) return fail(POLAR_ERR_ARG, "llr_max must be > 0");
    if (B > 0 && (!llr || !w)) return fail(POLAR_ERR_ARG, "NULL llr/w");
    const size_t need = wms_workspace_bytes(code, B, T);
    if (B > 0 && (!workspace || ws < need)) return fail(POLAR_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws, need);
    const DevCode* d = nullptr;
    if ((rc = code_slot(code, st, &d))) return rc;
    const size_t n = (size_t)log2i(code->N), N = (size_t)code->N;
    a = WMSArgs{};
    a.llr = llr;
    a.B = B;
    a.T = T;
    a.M = llr_max;
    a.w = w;
    a.store = static_cast<float*>(workspace);
    a.adj = a.store + (size_t)B * 2 * T * n * N;
    a.code = d;
    return POLAR_OK;
}

int wms_forward(const polar_code* code, const float* llr, int32_t B, int32_t T, float llr_max, const float* w,
                int32_t all_iters, float* llr_u, void* workspace, size_t ws, void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WMSArgs a;
    int rc = wms_common(code, llr, B, T, llr_max, w, workspace, ws, st, a);
    if (rc) return rc;
    if (B == 0) return POLAR_OK;
    if (!llr_u) return fail(POLAR_ERR_ARG, "NULL llr_u");
    a.all = all_iters ? 1 : 0;
    a.llr_u = llr_u;
    wms_forward_kernel<<<B, code->N / 2, 0, st>>>(a);
    POLAR_CUDA(cudaGetLastError());
    return POLAR_OK;
}

int wms_backward(const polar_code* code, const float* llr, int32_t B, int32_t T, float llr_max, const float* w,
                 int32_t all_iters, const float* grad_llr_u, float* grad_w, void* workspace, size_t ws,
                 void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WMSArgs a;
    int rc = wms_common(code, llr, B, T, llr_max, w, workspace, ws, st, a);
    if (rc) return rc;
    if (!grad_w) return fail(POLAR_ERR_ARG, "NULL grad_w");
    const size_t n = (size_t)log2i(code->N), N = (size_t)code->N;
    POLAR_CUDA(cudaMemsetAsync(grad_w, 0, (size_t)T * 2 * n * N * sizeof(float), st));
    if (B == 0) return POLAR_OK;
    if (!grad_llr_u) return fail(POLAR_ERR_ARG, "NULL grad_llr_u");
    a.all = all_iters ? 1 : 0;
    a.grad_u = grad_llr_u;
    a.grad_w = grad_w;
    wms_backward_kernel<<<B, code->N / 2, 0, st>>>(a);
    POLAR_CUDA(cudaGetLastError());
    return POLAR_OK;
}

// ------------------------------------------------------------------------------ mixed batches
namespace {

struct MixLayout {
    size_t counts, start, cursor, qnext, order, list, scratch, total;
};
MixLayout mix_layout(int ncodes, int B, size_t scratch_bytes)
{
    MixLayout m{};
    size_t o = kHeaderBytes;
    m.counts = o;
    o += sizeof(int) * ncodes;
    m.start = o;
    o += sizeof(int) * (ncodes + 1);
    m.cursor = o;
    o += sizeof(int) * ncodes;
    m.qnext = o;
    o += sizeof(int) * ncodes;
    o = align_up(o, 256);
    m.order = o;
    o = align_up(o + sizeof(int) * (size_t)std::max(B, 1), 256);
    m.list = o;
    o = align_up(o + sizeof(int) * (size_t)std::max(B, 1), 256);
    m.scratch = o;
    m.total = o + scratch_bytes;
    return m;
}

int mix_check(const polar_code* codes, int ncodes, int B, int L, int row_stride, int* max_row, int* warp_words,
              long long* slot_words)
{
    if (!codes || ncodes < 1 || ncodes > POLAR_MAX_MIX_CODES)
        return fail(POLAR_ERR_ARG, "ncodes = %d: must be in [1, %d]", ncodes, POLAR_MAX_MIX_CODES);
    if (B < 0) return fail(POLAR_ERR_ARG, "B < 0");
    int mr = 0, ww = 0;
    long long sw = 0;
    for (int c = 0; c < ncodes; ++c) {
        int rc = check_code(&codes[c]);
        if (rc) return rc;
        if (codes[c].N > POLAR_MAX_N_MIXED)
            return fail(POLAR_ERR_ARG, "mixed batches: N = %d > %d", codes[c].N, POLAR_MAX_N_MIXED);
        mr = std::max(mr, (codes[c].K - codes[c].crc_len + 7) / 8);
        if (L > 0) {
            // per-list words (+ the warp's 16 scratch words) and global slot of the CA-SCL launch's
            // list width (two lists per warp for L <= 8)
            const SCLPlan p = scl_plan(codes[c].N, L, false, scl_two_lists(L, false) ? 2 : 1);
            ww = std::max(ww, p.list_words + 16);
            sw = std::max(sw, p.slot_words);
        }
    }
    if (row_stride >= 0 && row_stride < mr) return fail(POLAR_ERR_ARG, "row_stride %d < %d bytes", row_stride, mr);
    if (max_row) *max_row = mr;
    if (warp_words) *warp_words = ww;
    if (slot_words) *slot_words = sw;
    return POLAR_OK;
}

std::mutex g_mix_mutex;
int g_mix_variant[2][12];  // [precision][log2 N] -> plan variant (0 = default)

int mix_default_variant(int n, int precision)
{
    std::lock_guard<std::mutex> lock(g_mix_mutex);
    const int v = g_mix_variant[precision][n];
    if (v) return v;  // 0 is the default plan of N = 128 as well: no entry needed
    return n == 7 ? 0 : n == 8 ? 1 : n == 9 ? 3 : n == 10 ? 5 : 6;
}

// Bucketing and the BP launch of a mixed batch (variants[c] per code); fail list into ws.
int mix_bp(const polar_code* codes, int ncodes, const DevCode* const* dcodes, const int* variants, const int32_t* code_of,
           const int64_t* llr_off, const float* llr, int B, int max_iters, float llr_max, int precision, uint8_t* bits,
           int row_stride, uint8_t* status, uint16_t* iters, char* ws, const MixLayout& ml, cudaStream_t st)
{
    int* hdr = reinterpret_cast<int*>(ws);
    int* counts = reinterpret_cast<int*>(ws + ml.counts);
    int* start = reinterpret_cast<int*>(ws + ml.start);
    int* cursor = reinterpret_cast<int*>(ws + ml.cursor);
    int* qnext = reinterpret_cast<int*>(ws + ml.qnext);
    int* order = reinterpret_cast<int*>(ws + ml.order);
    int* list = reinterpret_cast<int*>(ws + ml.list);
    POLAR_CUDA(cudaMemsetAsync(ws, 0, ml.order, st));
    POLAR_CUDA(mix_bucketing(code_of, B, ncodes, counts, start, cursor, order, st));
    MixedArgs m{};
    m.base.llr = llr;
    m.base.llr_off = reinterpret_cast<const long long*>(llr_off);
    m.base.B = B;
    m.base.max_iters = max_iters;
    m.base.llr_max = llr_max;
    m.base.bits = bits;
    m.base.status = status;
    m.base.iters = iters;
    m.base.fail_count = hdr + 1;
    m.base.fail_list = list;
    m.base.fail_total = hdr;
    m.base.row_bytes = row_stride;
    m.ncodes = ncodes;
    m.order = order;
    m.start = start;
    m.qnext = qnext;
    size_t smem = 0;
    bool packed = true;  // every code's CRC fits a 16-bit half of the syndrome word
    for (int c = 0; c < ncodes; ++c) {
        m.code[c] = dcodes[c];
        m.variant[c] = variants[c];
        smem = std::max(smem, mix_smem_bytes(variants[c]));
        packed = packed && codes[c].crc_len <= 16;
    }
    const void* fn = bp_mixed_fn(precision, packed);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "bp_mixed_kernel attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMixBlock, smem);
    if (e != cudaSuccess) return cuda_fail(e, "bp_mixed_kernel occupancy");
    const int grid = std::max(1, per_sm) * scl_sm_count();
    void* args[] = {&m};
    ProfScope prof(0, st);
    e = cudaLaunchKernel(fn, dim3(grid), dim3(kMixBlock), args, smem, st);
    return e == cudaSuccess ? POLAR_OK : cuda_fail(e, "bp_mixed_kernel launch");
}

int mix_prepare(const polar_code* codes, int ncodes, cudaStream_t st, const DevCode** dcodes)
{
    for (int c = 0; c < ncodes; ++c) {
        int rc = code_slot(&codes[c], st, &dcodes[c]);
        if (rc) return rc;
    }
    return POLAR_OK;
}

}  // namespace

size_t polar_mixed_workspace_bytes(const polar_code* codes, int32_t ncodes, int32_t B, int32_t L)
{
    int mr = 0, ww = 0;
    long long sw = 0;
    if (!valid_L(L) || mix_check(codes, ncodes, B, L, -1, &mr, &ww, &sw) != POLAR_OK) return 0;
    return mix_layout(ncodes, B, (size_t)scl_sm_count() * kSclWarpsPerSM * (size_t)sw * 4).total;
}

int hybrid_decode_mixed(const polar_code* codes, int32_t ncodes, const int32_t* code_of, const int64_t* llr_off,
                        const float* llr, int32_t B, int32_t max_iters, float llr_max, int32_t precision, int32_t L,
                        uint8_t* bits, int32_t row_stride, uint8_t* status, uint16_t* iters, void* workspace, size_t ws,
                        void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int mr = 0, ww = 0;
    long long sw = 0;
    if (!valid_L(L)) return fail(POLAR_ERR_ARG, "L = %d: must be 1, 2, 4, 8, 16 or 32", L);
    int rc = mix_check(codes, ncodes, B, L, row_stride, &mr, &ww, &sw);
    if (rc) return rc;
    if (bp_variant(precision)) return fail(POLAR_ERR_ARG, "mixed batches decode with min-sum and the CRC stop");
    if ((rc = check_bp_args(&codes[0], llr, B, max_iters, llr_max, precision, nullptr, 0, bits, status, iters))) return rc;
    if (B > 0 && (!code_of || !llr_off || !bits)) return fail(POLAR_ERR_ARG, "NULL code_of/llr_off/bits");
    const DevCode* dcodes[POLAR_MAX_MIX_CODES];
    if ((rc = mix_prepare(codes, ncodes, st, dcodes))) return rc;
    if (B == 0) return POLAR_OK;
    const size_t scratch = (size_t)scl_sm_count() * kSclWarpsPerSM * (size_t)sw * 4;
    const MixLayout ml = mix_layout(ncodes, B, scratch);
    if (!workspace || ws < ml.total) return fail(POLAR_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws, ml.total);
    int variants[POLAR_MAX_MIX_CODES];
    for (int c = 0; c < ncodes; ++c) variants[c] = mix_default_variant(log2i(codes[c].N), precision);
    char* base = static_cast<char*>(workspace);
    if ((rc = mix_bp(codes, ncodes, dcodes, variants, code_of, llr_off, llr, B, max_iters, llr_max, precision, bits,
                     row_stride, status, iters, base, ml, st)))
        return rc;
    int* hdr = reinterpret_cast<int*>(base);
    // The CRC failures sorted by code (into the BP bucketing's order array, free after BP), so that
    // the two half-warp lists of a CA-SCL warp mostly decode frames of one code; longest codes
    // first, so that the frames with the longest decoding latency do not start last.
    MixRank rank{};
    {
        int idx[POLAR_MAX_MIX_CODES];
        for (int c = 0; c < ncodes; ++c) idx[c] = c;
        std::stable_sort(idx, idx + ncodes, [&](int x, int y) { return codes[x].N > codes[y].N; });
        for (int r = 0; r < ncodes; ++r) rank.r[idx[r]] = r;
    }
    int* sorted = reinterpret_cast<int*>(base + ml.order);
    POLAR_CUDA(mix_sort_list(reinterpret_cast<int*>(base + ml.list), hdr + 1, B, code_of, ncodes, rank,
                             reinterpret_cast<int*>(base + ml.counts), reinterpret_cast<int*>(base + ml.start),
                             reinterpret_cast<int*>(base + ml.cursor), sorted, st));
    SCLArgs a{};
    a.llr = llr;
    a.B = B;
    a.L = L;
    a.bits = bits;
    a.status = status;
    a.code = dcodes[0];
    a.list = sorted;
    a.count = hdr + 1;
    a.next = hdr + 2;
    a.scratch = reinterpret_cast<float*>(base + ml.scratch);
    a.row_bytes = row_stride;
    a.code_of = code_of;
    a.llr_off = reinterpret_cast<const long long*>(llr_off);
    for (int c = 0; c < ncodes; ++c) a.codes[c] = dcodes[c];
    int nmax = 0;
    for (int c = 0; c < ncodes; ++c) nmax = std::max(nmax, codes[c].N);
    ProfScope prof(1, st);
    const cudaError_t e = scl_launch(a, nmax, L, st, ww, sw);
    return e == cudaSuccess ? POLAR_OK : cuda_fail(e, "scl_kernel launch (mixed)");
}

int polar_mixed_set_plan(int32_t log2n, int32_t nodes_per_thread, int32_t precision)
{
    if (precision != POLAR_FP32 && precision != POLAR_FP16) return fail(POLAR_ERR_ARG, "precision = %d", precision);
    int v = -1;
    for (int c = 0; c < kMixVariants; ++c)
        if (mix_variant_logn(c) == log2n && (1 << mix_variant_logr(c)) == nodes_per_thread) v = c;
    if (v < 0) return fail(POLAR_ERR_ARG, "no mixed BP plan with %d nodes per thread for N = 2^%d", nodes_per_thread, log2n);
    std::lock_guard<std::mutex> lock(g_mix_mutex);
    g_mix_variant[precision][log2n] = v;
    return POLAR_OK;
}

int polar_mixed_autotune(const polar_code* codes, int32_t ncodes, const int32_t* code_of, const int64_t* llr_off,
                         const float* llr, int32_t B, int32_t max_iters, float llr_max, int32_t precision, uint8_t* bits,
                         int32_t row_stride, uint8_t* status, uint16_t* iters, void* workspace, size_t ws, void* stream,
                         int32_t* chosen, float* best_ms, float* default_ms)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int mr = 0;
    int rc = mix_check(codes, ncodes, B, 0, row_stride, &mr, nullptr, nullptr);
    if (rc) return rc;
    if (bp_variant(precision)) return fail(POLAR_ERR_ARG, "mixed batches decode with min-sum and the CRC stop");
    if ((rc = check_bp_args(&codes[0], llr, B, max_iters, llr_max, precision, nullptr, 0, bits, status, iters))) return rc;
    if (B < 1 || !code_of || !llr_off || !bits) return fail(POLAR_ERR_ARG, "autotune needs a non-empty batch");
    const DevCode* dcodes[POLAR_MAX_MIX_CODES];
    if ((rc = mix_prepare(codes, ncodes, st, dcodes))) return rc;
    const MixLayout ml = mix_layout(ncodes, B, 0);
    if (!workspace || ws < ml.scratch) return fail(POLAR_ERR_WORKSPACE, "workspace %zu < %zu bytes", ws, ml.scratch);
    // plan options per length: the default first, then the alternative with b = 2 (4 nodes per
    // thread: twice as many threads per frame, half the registers, more column exchanges)
    int opts[13][2], nopt[13] = {}, pick[13] = {};
    bool present[13] = {};
    for (int c = 0; c < ncodes; ++c) present[log2i(codes[c].N)] = true;
    for (int n = 7; n <= 11; ++n) {
        opts[n][0] = n == 7 ? 0 : n == 8 ? 1 : n == 9 ? 3 : n == 10 ? 5 : 6;
        nopt[n] = 1;
        if (n == 8) opts[n][nopt[n]++] = 2;
        if (n == 9) opts[n][nopt[n]++] = 4;
        if (n == 10) opts[n][nopt[n]++] = 7;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    POLAR_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(POLAR_ERR_CUDA, "cudaEventCreate");
    }
    // BP time of the launch with the plans in pick[]: the least of two timed runs after one
    // untimed run (which also pays any one-time setup)
    auto time_plans = [&](float* out) -> int {
        int variants[POLAR_MAX_MIX_CODES];
        for (int c = 0; c < ncodes; ++c) {
            const int n = log2i(codes[c].N);
            variants[c] = opts[n][pick[n]];
        }
        float tmin = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaError_t e = cudaEventRecord(e0, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
            int r = mix_bp(codes, ncodes, dcodes, variants, code_of, llr_off, llr, B, max_iters, llr_max, precision,
                           bits, row_stride, status, iters, static_cast<char*>(workspace), ml, st);
            if (r) return r;
            float ms = 0;
            if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                return cuda_fail(e, "autotune timing");
            if (rep > 0) tmin = std::min(tmin, ms);
        }
        *out = tmin;
        return POLAR_OK;
    };
    // coordinate search: each length in turn keeps the fastest of its options, the others at their
    // current choice (the lengths share the launch, so each choice is timed on the whole batch)
    float base = 0.0f, best = 0.0f;
    rc = time_plans(&base);
    best = base;
    for (int n = 7; n <= 11 && !rc; ++n) {
        if (!present[n]) continue;
        for (int o = 1; o < nopt[n] && !rc; ++o) {
            const int keep = pick[n];
            pick[n] = o;
            float t = 0.0f;
            rc = time_plans(&t);
            if (!rc && t < best) best = t;
            else pick[n] = keep;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(g_mix_mutex);
        for (int n = 7; n <= 11; ++n)
            if (present[n]) g_mix_variant[precision][n] = opts[n][pick[n]];
    }
    if (chosen)
        for (int n = 0; n <= 12; ++n)
            chosen[n] = (n >= 7 && n <= 11 && present[n]) ? 1 << mix_variant_logr(opts[n][pick[n]]) : 0;
    if (best_ms) *best_ms = best;
    if (default_ms) *default_ms = base;
    return POLAR_OK;
}

int polar_profile_enable(int32_t on)
{
    g_prof.on = on != 0;
    return POLAR_OK;
}

int polar_profile_read(double* bp_ms, int32_t* bp_launches, double* scl_ms, int32_t* scl_launches)
{
    double t[2] = {0.0, 0.0};
    int cnt[2] = {0, 0};
    int rc = POLAR_OK;
    for (const ProfRecord& r : g_prof.recs) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess && rc == POLAR_OK) rc = cuda_fail(e, "polar_profile_read");
        t[r.kind] += ms;
        cnt[r.kind] += 1;
        g_prof.pool.push_back(r.start);
        g_prof.pool.push_back(r.stop);
    }
    g_prof.recs.clear();
    if (g_prof.err != cudaSuccess && rc == POLAR_OK)
        rc = cuda_fail(g_prof.err, "event creation or record while profiling (some launches went untimed)");
    g_prof.err = cudaSuccess;
    if (bp_ms) *bp_ms = t[0];
    if (bp_launches) *bp_launches = cnt[0];
    if (scl_ms) *scl_ms = t[1];
    if (scl_launches) *scl_launches = cnt[1];
    return rc;
}

int polar_pe_eval(int32_t op, const float* a, const float* b, float* out, int32_t n, void* stream)
{
    if (op != POLAR_PE_MINSUM && op != POLAR_PE_EXACT && op != POLAR_PE_EXACT_PACKED)
        return fail(POLAR_ERR_ARG, "op = %d", op);
    if (n < 0 || n > (1 << 30)) return fail(POLAR_ERR_ARG, "n = %d outside [0, 2^30]", n);
    if (n == 0) return POLAR_OK;
    if (!a || !b || !out) return fail(POLAR_ERR_ARG, "NULL a/b/out");
    const int threads = 256, work = op == POLAR_PE_EXACT_PACKED ? (n + 1) / 2 : n;
    pe_eval_kernel<<<(work + threads - 1) / threads, threads, 0, static_cast<cudaStream_t>(stream)>>>(op, a, b, out, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? POLAR_OK : cuda_fail(e, "pe_eval_kernel launch");
}

int polar_hybrid_fallback_count(const void* workspace, int32_t* out, void* stream)
{
    if (!workspace || !out) return fail(POLAR_ERR_ARG, "NULL workspace/out");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int v = 0;
    POLAR_CUDA(cudaMemcpyAsync(&v, workspace, sizeof(int), cudaMemcpyDeviceToHost, st));
    POLAR_CUDA(cudaStreamSynchronize(st));
    *out = v;
    return POLAR_OK;
}

}  // extern "C"

// ==================================================================================== no-alloc
// hybrid_decode_noalloc: the hybrid decoder for callers that cannot allocate device memory.  Its
// scratch (the two work counters and the list of frames that fall back to CA-SCL) lives in the
// file-scope array below, which every GPU that loads this library holds until the process exits.
namespace polar {

constexpr size_t kNoallocScratchBytes = kHeaderBytes + sizeof(int) * (size_t)POLAR_NOALLOC_MAX_FRAMES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mutex;
static std::vector<void*> g_noalloc_ptr;  // device address of g_noalloc_scratch, per device

// Device address of the static scratch on the current device.  Host code cannot pass the
// array's name to a kernel (on the host it names a host-side stand-in), so the address is looked
// up once per device with that device current.
static int noalloc_scratch(void** out)
{
    int dev = 0;
    POLAR_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if ((int)g_noalloc_ptr.size() <= dev) g_noalloc_ptr.resize(dev + 1, nullptr);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return POLAR_OK;
}

}  // namespace polar

extern "C" int hybrid_decode_noalloc(const polar_code* code, const float* llr, int32_t B, int32_t max_iters,
                                     float llr_max, int32_t precision, const void* wms_scales, int32_t wms_iters,
                                     int32_t L, uint8_t* bits, uint8_t* status, uint16_t* iters, void* stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_bp_args(code, llr, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status, iters);
    if (rc) return rc;
    if (!valid_L(L)) return fail(POLAR_ERR_ARG, "L = %d: must be 1, 2, 4, 8, 16 or 32", L);
    if (B > POLAR_NOALLOC_MAX_FRAMES)
        return fail(POLAR_ERR_ARG, "hybrid_decode_noalloc: B = %d exceeds the static limit of %d frames per call", B,
                    POLAR_NOALLOC_MAX_FRAMES);
    if (!scl_fits_smem(code->N, L))
        return fail(POLAR_ERR_ARG,
                    "hybrid_decode_noalloc: the CA-SCL list of N = %d, L = %d needs device scratch beyond the "
                    "static array; use hybrid_decode with a workspace",
                    code->N, L);
    const DevCode* d = nullptr;
    if ((rc = code_slot(code, st, &d))) return rc;
    if (B == 0) return POLAR_OK;
    void* scratch = nullptr;
    if ((rc = noalloc_scratch(&scratch))) return rc;
    char* base = static_cast<char*>(scratch);
    WsHeader* h = reinterpret_cast<WsHeader*>(base);
    int* list = reinterpret_cast<int*>(base + kHeaderBytes);
    // the array keeps the previous call's counters: they must start at zero
    POLAR_CUDA(cudaMemsetAsync(h, 0, sizeof(WsHeader), st));
    if ((rc = launch_bp(d, code, llr, B, max_iters, llr_max, precision, wms_scales, wms_iters, bits, status, iters,
                        nullptr, nullptr, &h->fail_count, list, st)))
        return rc;
    return launch_scl(d, code, llr, B, L, bits, status, list, &h->fail_count, &h->scl_next, nullptr, st);
}
