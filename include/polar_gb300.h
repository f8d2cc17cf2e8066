/*
 * polar_gb300.h -- C ABI of the GB300-native hybrid BP + CA-SCL polar decoder
 * (Cammerer, Leible, Stahl, Hoydis, ten Brink, arXiv 1609.09358).
 *
 * Conventions shared by every entry point
 *   - Pointers marked "device" must point to memory of the current CUDA device; "host" pointers
 *     to ordinary host memory.  The caller owns every buffer.  Decoder calls never allocate: the
 *     scratch they need comes from the caller's `workspace` (size from polar_workspace_bytes).
 *     The library keeps one small static device table of code descriptions (POLAR_MAX_CODES
 *     slots), filled on the first use of a code on a device.
 *   - State the library keeps across calls (none of it holds frame data):
 *       * that code table, and per device the cached device address of hybrid_decode_noalloc's
 *         static scratch array (about 256 KB, held by every GPU that loads the library);
 *       * per device, non-blocking streams it creates on first use and keeps until exit: two for
 *         hybrid_decode_host (a second compute stream, a copy stream) and POLAR_SCHED_BP_STREAMS + 1
 *         for hybrid_decode_scheduled (its BP streams and its CA-SCL stream); every call orders
 *         them after the caller's stream and the caller's stream after them, so they never run
 *         ahead of or behind the call;
 *       * one page-locked host array of per-chunk failure counts for hybrid_decode_scheduled
 *         (4 bytes per chunk, grown when a call needs more, kept until exit), under a lock;
 *       * per device and kernel, whether the kernel's shared-memory limit was raised;
 *       * the mixed BP plan table set by polar_mixed_autotune / polar_mixed_set_plan;
 *       * per host thread, the last error message and the profiling records of polar_profile_*
 *         (CUDA events, pooled).
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 *     stream).  The first call with a new code uploads that code's tables with a copy on
 *     `stream`; make it before any stream capture.
 *   - Return value: POLAR_OK (0) or a negative POLAR_ERR_*; polar_last_error() then gives a
 *     one-line message (thread-local).  The library never aborts the process.
 *   - Bit vectors are packed little-endian: bit p of a row is bit (p % 8) of byte p / 8.
 *     Rows are padded to whole bytes.
 *   - Index conventions (Sec. II, Fig. 1): x = u G with G = F^{(x)n}, F = [[1,0],[1,1]] in
 *     natural order (no bit reversal); information positions in ascending index order; the
 *     payload occupies the first P = K - crc_len of them and the CRC the last crc_len.
 *   - CRC: generator x^c + crc_poly, MSB first, register initialised to 0, no reflection, no
 *     final XOR (e.g. 0x07 for c = 8, 0x1021 for c = 16, 0x864CFB for c = 24).
 *   - Hard decisions are bit = (LLR < 0); frozen positions decode to 0.
 */
#ifndef POLAR_GB300_H
#define POLAR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- return codes */
#define POLAR_OK 0
#define POLAR_ERR_ARG (-1)       /* invalid argument (sizes, pointers, code description) */
#define POLAR_ERR_WORKSPACE (-2) /* workspace NULL or smaller than polar_workspace_bytes() */
#define POLAR_ERR_CUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define POLAR_ERR_TIMEOUT (-4)   /* a bounded device-side wait gave up */
#define POLAR_ERR_CAPACITY (-5)  /* more distinct codes in use than POLAR_MAX_CODES */

/* ---------------------------------------------------------------- per-frame status bytes */
#define POLAR_FRAME_BP_OK 1        /* BP met the CRC within max_iters */
#define POLAR_FRAME_SCL_OK 2       /* CA-SCL found a CRC-passing path */
#define POLAR_FRAME_SCL_CRC_FAIL 3 /* CA-SCL found none; the best-metric path is output */
#define POLAR_FRAME_BP_FAIL 4      /* bp_decode only: CRC not met after max_iters */

/* ---------------------------------------------------------------- options */
#define POLAR_FP32 0 /* BP messages in binary32 */
#define POLAR_FP16 1 /* BP messages in binary16, two frames per half2 register */
/* bp_decode only, OR-ed into precision: run exactly max_iters iterations (no CRC early stop);
 * the status still reports whether the CRC of the final hard decision holds. */
#define POLAR_FIXED_ITERS 0x100
/* BP variants of Sec. II-B, OR-ed into `precision` of bp_decode / hybrid_decode /
 * hybrid_decode_host / hybrid_decode_noalloc (POLAR_FP32 messages, no learned weights):
 *   POLAR_G_EXACT        the exact PE function g(a, b) = ln((1 + e^(a+b)) / (e^a + e^b)) instead of
 *                        min-sum; computed with fast exponentials and logarithms, so it matches an
 *                        exact evaluation to about 1e-6 per update, not to the bit
 *   POLAR_STOP_REENCODE  stop at the first iteration where HD(LLR(x)) equals the re-encoded
 *                        HD(LLR(u)) (x = u G) instead of when the CRC holds; a frame counts as
 *                        decoded (POLAR_FRAME_BP_OK, else CA-SCL in the hybrid) iff its CRC holds
 *                        when BP stops */
#define POLAR_G_EXACT 0x200
#define POLAR_STOP_REENCODE 0x400
/* OR into precision with learned weights: the caller vouches that every scale lies in [-1, 1].
 * Then |w g| <= |g| <= llr_max and the clip of the scaled term is skipped (the result is the
 * same); with POLAR_FP16 and max_iters <= wms_iters the two frames of a half2 register are also
 * kept on the same iteration (a frame that stops waits for its partner, and the pair takes its
 * next two frames together), so that one prepared scale serves both.  Each frame is decoded
 * exactly as without the flag; only which frames share a register, and when, differs.  Scales
 * outside [-1, 1] with this flag give unspecified results. */
#define POLAR_WMS_UNIT 0x800

#define POLAR_OP_BP 0
#define POLAR_OP_SCL 1
#define POLAR_OP_HYBRID 2
#define POLAR_OP_HYBRID_HOST 3
#define POLAR_OP_HYBRID_SCHED 4

#define POLAR_MIN_N 128
#define POLAR_MAX_N 4096
#define POLAR_MAX_N_MIXED 2048 /* mixed batches, learned weights and their training: N <= 2048 */
#define POLAR_MAX_L 32
#define POLAR_MAX_CODES 32

/* A polar code.  N = 2^n with POLAR_MIN_N <= N <= POLAR_MAX_N; K non-frozen positions of which
 * crc_len (0, 8, 16 or 24) carry the CRC, crc_len <= K <= N; frozen: HOST pointer to N bytes,
 * 1 = frozen (value 0), 0 = information.  scl_decided: NULL, or a HOST pointer to N bytes, 1 on
 * information positions that CA-SCL decides by each path's hard decision without branching the
 * list (the decision aiding of Sec. II-A, meant for the most reliable positions: see
 * polar_reliability); it changes scl_decode and the CA-SCL stage of the hybrid decoders, not BP.
 * The struct and the tables are read during the call only. */
typedef struct polar_code {
    int32_t N;
    int32_t K;
    int32_t crc_len;
    uint32_t crc_poly;
    const uint8_t* frozen;
    const uint8_t* scl_decided;
} polar_code;

/* Frozen-set construction (Sec. II: information on the K most reliable bit-channels; Sec. II-A
 * names the Bhattacharyya parameter as the reliability measure).  Host only, FP64, log domain:
 * ln Z0 = -design_rate * 10^(design_ebn0_db / 10); index bits are read MSB first, a 0 bit maps
 * Z -> 2Z - Z^2 and a 1 bit Z -> Z^2; the K indices with the smallest Z (ties: larger index) are
 * information positions.  frozen_out: host, N bytes; info_idx_out: host, K int32 ascending (may
 * be NULL).  Errors: POLAR_ERR_ARG for N not a power of two in [2, 2^20], K outside [0, N] or
 * design_rate <= 0. */
int polar_construct(int32_t N, int32_t K, double design_ebn0_db, double design_rate,
                    uint8_t* frozen_out, int32_t* info_idx_out);

/* Bhattacharyya parameters of the construction (Sec. II-A): ln Z of every bit-channel at the
 * design point, computed as in polar_construct (smaller = more reliable).  Host only.
 *   lnz_out: host, N doubles.  POLAR_ERR_ARG for N not a power of two in [2, 2^20], a bad design
 *   point or a NULL output. */
int polar_reliability(int32_t N, double design_ebn0_db, double design_rate, double* lnz_out);

/* Systematic CRC + polar encoder (Sec. II, x = u G; CRC-aided construction of Sec. II-A).
 * payload: device, [B][ceil(P/8)] packed payload bits; codeword: device, [B][N/8] packed code
 * bits.  B >= 0 (B = 0 is a no-op). */
int polar_encode(const polar_code* code, const uint8_t* payload, int32_t B, uint8_t* codeword,
                 void* stream);

/* Seeded workload generator (not part of the paper's method): payload bits and BPSK-over-AWGN
 * channel LLRs from the counter-based generator Philox4x32-10 (Salmon et al., SC'11).  Key =
 * (seed low, seed high); counter = (block, frame low, stream, frame high) for frame index
 * frame0 + b.  polar_random_payload: stream 0, bit p of a frame is bit p % 32 of word p / 32.
 * polar_awgn_llr: stream 1, Box-Muller on 24-bit uniforms; llr = 2 (1 - 2x + sigma z) / sigma^2
 * (the LLR definition of Sec. II-A).  payload: device [B][ceil(P/8)]; codeword: device [B][N/8]
 * packed; llr: device float [B][N]; sigma_per_frame: NULL (every frame uses sigma) or device
 * float [B]. */
int polar_random_payload(int32_t B, int32_t P, uint64_t seed, uint64_t frame0, uint8_t* payload,
                         void* stream);
int polar_awgn_llr(const uint8_t* codeword, int32_t B, int32_t N, float sigma,
                   const float* sigma_per_frame, uint64_t seed, uint64_t frame0, float* llr,
                   void* stream);

/* Min-sum belief propagation with CRC early stop (Sec. II-B; PE of Fig. 2 on the graph of
 * Fig. 1).  One iteration updates the R messages of columns 2..n+1, then the L messages of
 * columns n..1, each PE computing
 *   R_out1 = g(R_in1, L_in2 + R_in2), R_out2 = g(R_in1, L_in1) + R_in2,
 *   L_out1 = g(L_in1, L_in2 + R_in2), L_out2 = g(R_in1, L_in1) + L_in2,
 * g(a, b) = sign(a) sign(b) min(|a|, |b|); every message and the channel LLRs are clipped to
 * [-llr_max, llr_max] (NaN channel values read as 0).  Init L_{i,n+1} = LLR(y_i),
 * R_{i,1} = llr_max f_i.  After each iteration the hard decision of LLR(u_i) = L_{i,1} + R_{i,1}
 * is CRC-checked and the frame stops when it passes.
 *   llr: device float [B][N].  max_iters >= 1.  llr_max > 0.
 *   precision: POLAR_FP32 (bit-exact with a binary32 reference) or POLAR_FP16 (binary16
 *     messages, llr_max <= 32768), optionally | POLAR_FIXED_ITERS (run max_iters iterations
 *     whatever the CRC), and for POLAR_FP32 without weights | POLAR_G_EXACT and/or
 *     | POLAR_STOP_REENCODE (the variants of Sec. II-B described with those flags).
 *   wms_scales: NULL, or the learned weights of a weighted min-sum BP as prepared by
 *     wms_prepare for this code, wms_iters and precision (device, 16-byte aligned): each g term
 *     is multiplied by its scale before the clip; iterations t >= wms_iters run unweighted.
 *   bits: device [B][ceil(P/8)] decided payload.  status: device [B] POLAR_FRAME_BP_OK or
 *     POLAR_FRAME_BP_FAIL.  iters: device uint16 [B], iterations run.
 *   llr_u, llr_x: NULL or device float [B][N], the final LLR(u) and LLR(x).
 *   workspace: may be NULL (polar_workspace_bytes(.., POLAR_OP_BP) is 0). */
int bp_decode(const polar_code* code, const float* llr, int32_t B, int32_t max_iters,
              float llr_max, int32_t precision, const void* wms_scales, int32_t wms_iters,
              uint8_t* bits, uint8_t* status, uint16_t* iters, float* llr_u, float* llr_x,
              void* workspace, size_t ws_bytes, void* stream);

/* CRC-aided successive cancellation list decoding (Sec. II-A; list decoding of Tal and Vardy).
 * Min-sum f, exact g, path metric m' = m + |lambda| [b != HD(lambda)]; at an information bit the
 * L smallest of the 2L candidates by (m', 2 path + b) survive (the paper's pruned pseudo sort
 * with a total order) and are renumbered in ascending candidate index; after the last bit the
 * first path, in (metric, path index) order, whose CRC passes is output.
 *   llr: device float [B][N].  L in {1, 2, 4, 8, 16, 32}.
 *   bits: device [B][ceil(P/8)]; status: device [B] POLAR_FRAME_SCL_OK / _SCL_CRC_FAIL.
 *   workspace: device, >= polar_workspace_bytes(code, B, L, POLAR_OP_SCL) bytes. */
int scl_decode(const polar_code* code, const float* llr, int32_t B, int32_t L, uint8_t* bits,
               uint8_t* status, void* workspace, size_t ws_bytes, void* stream);

/* Hybrid decoder (Sec. III, Fig. 3): BP as in bp_decode on every frame; the frames whose CRC
 * still fails after max_iters are compacted on the device and decoded by CA-SCL as in
 * scl_decode.  status: POLAR_FRAME_BP_OK, _SCL_OK or _SCL_CRC_FAIL; iters: BP iterations.
 *   workspace: device, >= polar_workspace_bytes(code, B, L, POLAR_OP_HYBRID) bytes. */
int hybrid_decode(const polar_code* code, const float* llr, int32_t B, int32_t max_iters,
                  float llr_max, int32_t precision, const void* wms_scales, int32_t wms_iters,
                  int32_t L, uint8_t* bits, uint8_t* status, uint16_t* iters, void* workspace,
                  size_t ws_bytes, void* stream);

/* Learned weights for decoding (the configurations' learned variant; not in the paper).
 * w: device float [wms_iters][2][n][N]; entry [t][0][s-1][i] scales the g term of the R message
 * written to node i by PE stage s in iteration t, entry [t][1][s-1][i] that of the L message.
 * wms_prepare rewrites them into the decoder's per-thread register order, in the message
 * precision (binary16 values rounded to nearest even for POLAR_FP16), into `prepared` (device,
 * 16-byte aligned, >= wms_prepared_bytes(code, wms_iters, precision) bytes, owned by the caller).
 * The prepared buffer is then passed as wms_scales to bp_decode / hybrid_decode with the same
 * code, wms_iters and precision; preparing once and decoding many batches reads each scale with
 * one vector load per thread and stage.  wms_prepared_bytes returns 0 on invalid arguments.
 * Errors: POLAR_ERR_ARG (invalid code, N outside [128, POLAR_MAX_N_MIXED], wms_iters < 1, NULL or misaligned
 * pointer), POLAR_ERR_WORKSPACE (buffer too small), POLAR_ERR_CUDA. */
size_t wms_prepared_bytes(const polar_code* code, int32_t wms_iters, int32_t precision);
int wms_prepare(const polar_code* code, const float* w, int32_t wms_iters, int32_t precision,
                void* prepared, size_t bytes, void* stream);

/* Training of the learned weighted min-sum BP (the configurations' learned variant; not in the
 * paper).  wms_forward runs T iterations of the weighted BP of bp_decode (no early stop) and
 * writes LLR(u) = L_{.,1} + R_{.,1}, storing every message in the workspace: of the last
 * iteration into llr_u [B][N] (all_iters = 0), or of every iteration into llr_u [T][B][N]
 * (all_iters = 1, for a loss summed over iterations).  wms_backward, given dLoss/dLLR(u) in the
 * same shape, writes dLoss/dw for w[T][2][n][N] (overwritten, summed over the batch) by a
 * hand-written reverse sweep through the stored messages (subgradients of min and clip).  Call
 * wms_backward after wms_forward with the same llr, w, all_iters and workspace.  llr, w, llr_u,
 * grad_llr_u, grad_w: device.  workspace: device, >= wms_workspace_bytes(code, B, T).
 * 1 <= T <= 1000. */
size_t wms_workspace_bytes(const polar_code* code, int32_t B, int32_t T);
int wms_forward(const polar_code* code, const float* llr, int32_t B, int32_t T, float llr_max,
                const float* w, int32_t all_iters, float* llr_u, void* workspace, size_t ws_bytes,
                void* stream);
int wms_backward(const polar_code* code, const float* llr, int32_t B, int32_t T, float llr_max,
                 const float* w, int32_t all_iters, const float* grad_llr_u, float* grad_w,
                 void* workspace, size_t ws_bytes, void* stream);

/* Mixed batch (the configurations' mixed workload; not in the paper): frames of up to
 * POLAR_MAX_MIX_CODES codes of different lengths and rates in one batch.  Frames are bucketed by
 * code on the device, then one persistent BP launch decodes all of them (a CTA works on one code
 * at a time and moves to the next when that code's queue is empty) and one CA-SCL launch decodes
 * every frame whose CRC failed, each with its own code (failures sorted by code first).  Nothing waits for the host, so the call
 * can be captured in a CUDA graph once each code has been used (code tables uploaded) and
 * polar_mixed_autotune has run.  Results equal hybrid_decode of each frame with its own code.
 *   codes: host array of ncodes code descriptions.  code_of: device int32 [B], code of each frame
 *   (a frame with a code id outside [0, ncodes) is not decoded and its outputs are not written).
 *   llr_off: device int64 [B], element offset of each frame's LLR row in llr (device float).
 *   bits: device [B][row_stride], row_stride >= ceil(P/8) of every code; status, iters: [B].
 *   workspace: device, >= polar_mixed_workspace_bytes(codes, ncodes, B, L). */
#define POLAR_MAX_MIX_CODES 32
size_t polar_mixed_workspace_bytes(const polar_code* codes, int32_t ncodes, int32_t B, int32_t L);
int hybrid_decode_mixed(const polar_code* codes, int32_t ncodes, const int32_t* code_of,
                        const int64_t* llr_off, const float* llr, int32_t B, int32_t max_iters,
                        float llr_max, int32_t precision, int32_t L, uint8_t* bits,
                        int32_t row_stride, uint8_t* status, uint16_t* iters, void* workspace,
                        size_t ws_bytes, void* stream);
/* Autotuner of the mixed BP launch: for each block length of the batch that has two BP thread
 * plans (256, 512 and 1024: 8 or 4 nodes per thread, i.e. one frame on half or twice as many
 * threads, so twice or half as many frames per CTA) it times the BP launch on this batch with each
 * choice, one length at a time (the others at their current choice), and keeps the fastest for
 * later hybrid_decode_mixed calls of the same precision (a table inside the library, per
 * precision).  Synchronises `stream`; overwrites the outputs.  Arguments as in
 * hybrid_decode_mixed.  chosen (host, may be NULL): 13 entries indexed by log2 N, the nodes per
 * thread chosen for each length in the batch (0 for the others); *best_ms the BP time of the
 * chosen plans, *default_ms that of the default plans (8 nodes per thread from N = 256 on). */
int polar_mixed_autotune(const polar_code* codes, int32_t ncodes, const int32_t* code_of,
                         const int64_t* llr_off, const float* llr, int32_t B, int32_t max_iters,
                         float llr_max, int32_t precision, uint8_t* bits, int32_t row_stride,
                         uint8_t* status, uint16_t* iters, void* workspace, size_t ws_bytes,
                         void* stream, int32_t* chosen, float* best_ms, float* default_ms);

/* Sets the mixed BP plan of one block length by hand (as polar_mixed_autotune would): N = 2^log2n
 * decoded with nodes_per_thread nodes per thread (8 or 4 for N = 256, 512 and 1024; 4 for N = 128;
 * 8 for N = 2048) in later hybrid_decode_mixed calls of this precision.  POLAR_ERR_ARG for a plan
 * that does not exist. */
int polar_mixed_set_plan(int32_t log2n, int32_t nodes_per_thread, int32_t precision);

/* hybrid_decode on frames that live in host memory (not a step of the paper; its Sec. III
 * rejects moving SCL to the CPU because of transfer latency, which is what this hides).  The
 * LLRs are copied to the device in chunks (4096 and 8192 frames, then POLAR_HOST_CHUNK) on a
 * library-owned copy stream; each chunk's BP launch starts as soon as its own copy has landed (chunks
 * alternating between `stream` and a second library-owned stream, so one chunk's last frames
 * overlap the next), all chunks append to one fail list, one CA-SCL launch decodes every frame BP
 * failed, and one copy per output brings the results back.  The call is ordered after earlier
 * work on `stream` and later work on `stream` is ordered after it; it returns before completion
 * when the host buffers are page-locked.  The workspace holds the whole batch (about 4N bytes per
 * frame plus the hybrid workspace).
 *   llr_host: host float [B][N]; bits_host [B][ceil(P/8)], status_host [B], iters_host [B]:
 *   host.  wms_scales: device or NULL.  workspace: device, >= polar_workspace_bytes(code, B, L,
 *   POLAR_OP_HYBRID_HOST). */
#define POLAR_HOST_CHUNK 16384
int hybrid_decode_host(const polar_code* code, const float* llr_host, int32_t B, int32_t max_iters,
                       float llr_max, int32_t precision, const void* wms_scales, int32_t wms_iters,
                       int32_t L, uint8_t* bits_host, uint8_t* status_host, uint16_t* iters_host,
                       void* workspace, size_t ws_bytes, void* stream);

/* Host-scheduled hybrid decoding: the scheduling of Fig. 3 (Sec. III), kept to measure what it
 * costs against hybrid_decode's two stream-ordered launches.  The batch is cut into chunks of
 * `chunk` frames.  While fewer than POLAR_SCHED_BP_STREAMS chunks are in BP, the host starts the
 * next chunk's BP launch on a free library-owned stream ("enough buffer space"); it polls those
 * launches, and when one has finished it reads that chunk's count of CRC failures ("BP finished");
 * whenever failed frames are waiting and the CA-SCL stream is idle, it launches CA-SCL on them
 * ("start idle SCL decoders": one launch per waiting chunk, on one library-owned stream).  Failed
 * frames are not copied: BP lists their indices and CA-SCL reads their LLR rows in place.  The call
 * returns once the last CA-SCL launch is issued (the host has seen every BP launch finish); work
 * issued later on `stream` is ordered after all of it.  Results equal hybrid_decode's.
 *   llr, bits, status, iters: device, as for hybrid_decode.  chunk: frames per BP launch, >= 256.
 *   workspace: device, >= polar_workspace_bytes(code, B, L, POLAR_OP_HYBRID_SCHED) bytes.
 *   Errors: as hybrid_decode; POLAR_ERR_ARG for chunk < 256; POLAR_ERR_TIMEOUT if a launch has
 *   not finished 600 s after the host last saw progress. */
#define POLAR_SCHED_BP_STREAMS 3
int hybrid_decode_scheduled(const polar_code* code, const float* llr, int32_t B, int32_t max_iters,
                            float llr_max, int32_t precision, const void* wms_scales, int32_t wms_iters,
                            int32_t L, int32_t chunk, uint8_t* bits, uint8_t* status, uint16_t* iters,
                            void* workspace, size_t ws_bytes, void* stream);

/* Kernel timing for measurement (not a step of the paper).  While enabled on the calling host
 * thread, every decoder call brackets its BP and SCL kernel launches with CUDA events on the
 * launch stream.  polar_profile_read waits for the recorded events, returns the summed device
 * time in milliseconds and the launch count of each kernel kind, and clears the record. */
int polar_profile_enable(int32_t on);
int polar_profile_read(double* bp_ms, int32_t* bp_launches, double* scl_ms, int32_t* scl_launches);

/* The PE function of the BP kernels (Sec. II-B, Fig. 2), elementwise, for checking it against a
 * reference (not a decoding step): out[i] = g(a[i], b[i]), unclipped (the decoders clip it).
 *   op: POLAR_PE_MINSUM (sign(a) sign(b) min(|a|, |b|), exact in binary32), POLAR_PE_EXACT
 *   (ln((1 + e^(a+b)) / (e^a + e^b)) with the fast exponential and logarithm, the scalar form) or
 *   POLAR_PE_EXACT_PACKED (the same arithmetic as two-lane packed instructions, as the FP32 BP
 *   kernels evaluate it; elements 2i and 2i+1 are one pair).  a, b, out: device float [n],
 *   0 <= n <= 2^30.  Asynchronous on `stream`.  POLAR_ERR_ARG for an unknown op, n outside that
 *   range or NULL pointers. */
#define POLAR_PE_MINSUM 0
#define POLAR_PE_EXACT 1
#define POLAR_PE_EXACT_PACKED 2
int polar_pe_eval(int32_t op, const float* a, const float* b, float* out, int32_t n, void* stream);

/* Issue-rate microbenchmark (measurement only, not a step of the paper): the throughput of one
 * instruction the BP kernels' roofline rests on, as results of one lane (an f16x2 instruction
 * counts once) per SM per SM clock, averaged over the SMs.  32 warps per SM each run 8
 * independent dependency chains of the instruction; every CTA times its loop with clock64().
 *   op: one of POLAR_RATE_*.  iters >= 1: rounds of the 8 chains per thread (4096 takes about a
 *   millisecond).  scratch: device, >= polar_pipe_rate_scratch_bytes() bytes, owned by the caller.
 *   Synchronises `stream`.  POLAR_ERR_ARG for an unknown op, iters < 1 or NULL pointers,
 *   POLAR_ERR_WORKSPACE for a short scratch.  polar_pipe_rate_scratch_bytes returns 0 if the
 *   current device cannot be queried. */
#define POLAR_RATE_MINXORSIGN_F32 0   /* min.xorsign.abs.f32: the min-sum g and the clip */
#define POLAR_RATE_MINXORSIGN_F16X2 1 /* min.xorsign.abs.f16x2 */
#define POLAR_RATE_ADD_F32 2          /* add.rn.f32 */
#define POLAR_RATE_ADD_F16X2 3        /* add.rn.f16x2 */
#define POLAR_RATE_MUL_F16X2 4        /* mul.rn.f16x2: the learned scales of the half2 kernels */
#define POLAR_RATE_MIN_F32 5          /* min.f32 */
#define POLAR_RATE_EX2_F32 6          /* ex2.approx.ftz.f32: the exact PE function */
#define POLAR_RATE_LG2_F32 7          /* lg2.approx.ftz.f32 */
#define POLAR_RATE_PRMT 8             /* prmt.b32: byte permute (pairing of half2 values) */
size_t polar_pipe_rate_scratch_bytes(void);
int polar_pipe_rate(int32_t op, int32_t iters, void* scratch, size_t scratch_bytes, double* per_sm_clock,
                    void* stream);

/* hybrid_decode without any device allocation (the paper has no counterpart: this exists for
 * callers that cannot allocate device memory -- for instance a receive chain that must never call
 * cudaMalloc once running, because an allocation can synchronise the device and take unbounded
 * time, or a plug-in whose host application owns and budgets all device memory).  It decodes like
 * hybrid_decode but takes no workspace: its scratch (two counters and the list of frames that go
 * to CA-SCL) is one static device array of about 256 KB inside this library, which every GPU that
 * loads the library holds until the process exits.
 *   Limits: B <= POLAR_NOALLOC_MAX_FRAMES, and one frame's CA-SCL list (its LLR and
 *   partial-sum arrays, about 4 L N bytes) must fit in 80 KiB of shared memory, e.g. N = 1024
 *   with L <= 16; larger requests return POLAR_ERR_ARG with a message.
 *   The first call on a device looks up the array's device address (and, like every first use of
 *   a code, uploads the code tables); make that first call before any stream capture.
 *   All calls share the array and it keeps the last call's contents; the counters are cleared on
 *   `stream` at the start of every call.  Calls that overlap on the GPU (different streams, or
 *   different host threads) race on the array and must be serialised by the caller.
 *   Nothing here calls cudaMalloc, cudaFree or any allocating routine.  Other arguments as in
 *   hybrid_decode. */
#define POLAR_NOALLOC_MAX_FRAMES 65536
int hybrid_decode_noalloc(const polar_code* code, const float* llr, int32_t B, int32_t max_iters,
                          float llr_max, int32_t precision, const void* wms_scales,
                          int32_t wms_iters, int32_t L, uint8_t* bits, uint8_t* status,
                          uint16_t* iters, void* stream);

/* Device workspace needed by an operation (op = POLAR_OP_*) on B frames with list size L
 * (ignored for POLAR_OP_BP).  Returns 0 on invalid arguments as well as when none is needed. */
size_t polar_workspace_bytes(const polar_code* code, int32_t B, int32_t L, int32_t op);

/* Number of frames that the last hybrid_decode on `workspace` sent to CA-SCL, copied to *out
 * (host) after synchronising `stream`. */
int polar_hybrid_fallback_count(const void* workspace, int32_t* out, void* stream);

/* Message of the last failed call on this host thread ("" if none). */
const char* polar_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* POLAR_GB300_H */
