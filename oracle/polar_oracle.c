/*
 * polar_oracle.c -- plain, slow CPU reference for the hybrid BP + CA-SCL polar decoder of
 * Cammerer et al., "Combining Belief Propagation and Successive Cancellation List Decoding of
 * Polar Codes on a GPU Platform" (arXiv 1609.09358).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code with the CUDA decoder: it is written
 * straight from the paper's definitions, one frame at a time, with full message arrays and eager
 * path copies, and nothing is blocked, fused or reordered.
 *
 * Conventions where the paper is silent (each is a reading, not a paper fact):
 *   - natural-order transform x = u G, G = F^{(x)n}, F = [[1,0],[1,1]] (Sec. II, Fig. 1):
 *     G[i][j] = 1 iff the bits of j are a subset of the bits of i;
 *   - info positions in ascending index order; payload in the first P = K - c of them, the c CRC
 *     bits in the last c (Sec. II; CRC-aided list decoding and the rate (k-c)/N in Sec. II-A);
 *   - CRC: plain polynomial division, MSB-first, register starts at 0, no reflection, no final XOR;
 *   - hard decision bit = (LLR < 0), frozen positions forced to 0;
 *   - every computed BP message is clipped to [-LLR_max, +LLR_max] (Sec. II-B), channel LLRs too;
 *   - SCL: min-sum f, exact g, hard-decision path-metric penalty |lambda| [b != HD(lambda)],
 *     candidates ordered by (metric, 2*path + bit), survivors renumbered by ascending candidate
 *     index, final choice = first CRC-passing path in (metric, path index) order.
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#define _DEFAULT_SOURCE /* M_LN2 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <fenv.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------------ */
/* Code construction (Sec. II: information on the k most reliable bit-channels; Sec. II-A     */
/* names the Bhattacharyya parameter as the reliability measure).                             */
/* ------------------------------------------------------------------------------------------ */

/* ln Z of bit-channel i for a BI-AWGN channel with ln Z0 = -R * Eb/N0 (linear).  The index is
 * read MSB first: the MSB is the first (channel-side) combining step of Fig. 1.  A 0 bit takes the
 * "minus" channel Z -> 2Z - Z^2, a 1 bit the "plus" channel Z -> Z^2.  Computed in the log domain
 * so that Z^(2^n) does not underflow.  For the minus step, ln(2Z - Z^2) = ln Z + ln(2 - Z) when
 * Z <= 1/2, and ln(1 - (1 - Z)^2) with 1 - Z = -expm1(ln Z) when Z > 1/2, where the first form
 * would round to ln Z > 0. */
double or_bhattacharyya_lnz(int n, int i, double lnz0)
{
    double lnz = lnz0;
    for (int level = n - 1; level >= 0; --level) {
        int bit = (i >> level) & 1;
        if (bit) {
            lnz = 2.0 * lnz;
        } else if (lnz <= -M_LN2) {
            lnz = lnz + log(2.0 - exp(lnz));
        } else {
            double one_minus_z = -expm1(lnz);
            lnz = log1p(-(one_minus_z * one_minus_z));
        }
    }
    return lnz;
}

/* Frozen set: the K indices with the smallest Z are information positions.  Ties in Z go to the
 * larger index.  frozen[i] = 1 for frozen, 0 for information; info_idx = ascending info indices.
 * Returns 0, or -1 on bad arguments. */
int or_construct(int N, int K, double design_ebn0_db, double design_rate,
                 unsigned char* frozen, int* info_idx, double* lnz_out)
{
    int n = 0;
    while ((1 << n) < N) ++n;
    if ((1 << n) != N || K < 0 || K > N || design_rate <= 0.0) return -1;
    double lnz0 = -design_rate * pow(10.0, design_ebn0_db / 10.0);
    double* lnz = (double*)malloc(sizeof(double) * N);
    for (int i = 0; i < N; ++i) lnz[i] = or_bhattacharyya_lnz(n, i, lnz0);
    if (lnz_out) memcpy(lnz_out, lnz, sizeof(double) * N);
    /* selection by repeated minimum: plain O(N*K) */
    for (int i = 0; i < N; ++i) frozen[i] = 1;
    for (int k = 0; k < K; ++k) {
        int best = -1;
        for (int i = 0; i < N; ++i) {
            if (!frozen[i]) continue;
            if (best < 0 || lnz[i] < lnz[best] || (lnz[i] == lnz[best] && i > best)) best = i;
        }
        frozen[best] = 0;
    }
    int k = 0;
    for (int i = 0; i < N; ++i)
        if (!frozen[i]) info_idx[k++] = i;
    free(lnz);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* CRC (Sec. II-A: c CRC bits appended to the information, R_crc = (k - c)/N).                */
/* ------------------------------------------------------------------------------------------ */

/* Remainder of the polynomial division of m(x) by g(x) = x^c + poly(x), all coefficients in
 * GF(2), the first bit being the highest power.  Written as schoolbook long division over a bit
 * array.  rem_out gets c bits, highest power first. */
void or_poly_mod(const unsigned char* m, int nbits, unsigned poly, int c, unsigned char* rem_out)
{
    unsigned char* work = (unsigned char*)malloc((size_t)nbits + 1);
    unsigned char* g = (unsigned char*)malloc((size_t)c + 1);
    memcpy(work, m, (size_t)nbits);
    g[0] = 1;
    for (int k = 1; k <= c; ++k) g[k] = (unsigned char)((poly >> (c - k)) & 1u);
    for (int i = 0; i + c < nbits; ++i) {
        if (!work[i]) continue;
        for (int k = 0; k <= c; ++k) work[i + k] ^= g[k];
    }
    for (int k = 0; k < c; ++k) rem_out[k] = (nbits - c + k >= 0) ? work[nbits - c + k] : 0;
    free(work);
    free(g);
}

/* CRC of a message: remainder of m(x) * x^c divided by g(x). */
void or_crc(const unsigned char* msg, int nbits, unsigned poly, int c, unsigned char* crc_out)
{
    unsigned char* m = (unsigned char*)calloc((size_t)nbits + (size_t)c + 1, 1);
    memcpy(m, msg, (size_t)nbits);
    or_poly_mod(m, nbits + c, poly, c, crc_out);
    free(m);
}

/* 1 if the K bits (payload followed by its CRC) form a valid CRC codeword. */
int or_crc_check(const unsigned char* bits, int nbits, unsigned poly, int c)
{
    if (c == 0) return 1;
    unsigned char rem[32];
    or_poly_mod(bits, nbits, poly, c, rem);
    for (int k = 0; k < c; ++k)
        if (rem[k]) return 0;
    return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Encoder (Sec. II, Fig. 1): x = u G with G = F^{(x)n}.                                     */
/* ------------------------------------------------------------------------------------------ */

/* Entry (i, j) of G = F^{(x)n}: the product over bit positions of F[i_b][j_b]; F[0][1] = 0 is the
 * only zero entry of F, so G[i][j] = 1 iff no bit position has i_b = 0 and j_b = 1. */
int or_generator_entry(int i, int j)
{
    return (j & ~i) == 0;
}

/* x_j = XOR over i of u_i G[i][j], the plain O(N^2) matrix-vector product over GF(2). */
void or_polar_transform(const unsigned char* u, int N, unsigned char* x)
{
    for (int j = 0; j < N; ++j) {
        unsigned char acc = 0;
        for (int i = 0; i < N; ++i) acc ^= (unsigned char)(u[i] & or_generator_entry(i, j));
        x[j] = acc;
    }
}

/* The encoder circuit of Fig. 1: n stages of XOR butterflies.  Stage s (s = 1..n, counted from
 * the u side) XORs node j + d into node j for every j with bit s-1 clear, d = 2^(s-1).  O(N log N)
 * (Sec. II); pinned against the matrix definition above. */
void or_encode_circuit(const unsigned char* u, int N, unsigned char* x)
{
    memcpy(x, u, (size_t)N);
    for (int d = 1; d < N; d <<= 1)
        for (int j = 0; j < N; ++j)
            if (!(j & d)) x[j] ^= x[j + d];
}

/* u vector of one frame: payload into the first P info positions, CRC of the payload into the
 * last c info positions, zeros on frozen positions. */
void or_build_u(const unsigned char* payload, int N, int K, const int* info_idx,
                unsigned poly, int c, unsigned char* u)
{
    int P = K - c;
    unsigned char crc[32];
    memset(u, 0, (size_t)N);
    or_crc(payload, P, poly, c, crc);
    for (int k = 0; k < P; ++k) u[info_idx[k]] = payload[k] & 1;
    for (int k = 0; k < c; ++k) u[info_idx[P + k]] = crc[k];
}

/* Batch encoder: payload [B][P] (one byte per bit) -> codeword [B][N] (one byte per bit), by the
 * Fig. 1 circuit (pinned equal to the matrix definition). */
void or_encode_batch(const unsigned char* payload, int B, int N, int K, const int* info_idx,
                     unsigned poly, int c, unsigned char* x)
{
    int P = K - c;
    unsigned char* u = (unsigned char*)malloc((size_t)N);
    for (int b = 0; b < B; ++b) {
        or_build_u(payload + (size_t)b * P, N, K, info_idx, poly, c, u);
        or_encode_circuit(u, N, x + (size_t)b * N);
    }
    free(u);
}

/* BPSK over AWGN (Sec. II-A LLR definition, LLR(y) = ln P(y|0)/P(y|1)): s = 1 - 2x,
 * y = s + sigma * noise, LLR = 2 y / sigma^2.  Computed in FP64, rounded once to FP32. */
void or_channel_llr(const unsigned char* x, const double* noise, long long count, double sigma,
                    float* llr_out)
{
    for (long long i = 0; i < count; ++i) {
        double s = 1.0 - 2.0 * (double)(x[i] & 1);
        double y = s + sigma * noise[i];
        llr_out[i] = (float)(2.0 * y / (sigma * sigma));
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Round to IEEE 754 binary16 (round to nearest, ties to even), returned as a float that holds  */
/* the exact half value.  Used to emulate the half-precision BP messages: a sum of two binary16  */
/* values formed in binary32 and then rounded to binary16 is the correctly rounded binary16 sum, */
/* because 24 >= 2*11 + 2 (double rounding is innocuous at that precision gap).               */
/* ------------------------------------------------------------------------------------------ */
float or_round_half(float x)
{
    double ax = fabs((double)x);
    if (ax == 0.0 || isnan(x)) return x;
    if (ax >= 65520.0) return copysignf(INFINITY, x);
    int e;
    frexp(ax, &e);                           /* ax = m 2^e, m in [0.5, 1) */
    int q = (e - 1 >= -14) ? (e - 11) : -24; /* exponent of the binary16 ulp at this magnitude */
    double r = nearbyint(ldexp(ax, -q));     /* default rounding mode: nearest, ties to even */
    return (float)copysign(ldexp(r, q), (double)x);
}

/* BP modes (or_bp_decode's `mode`, or_hybrid_decode_batch's `bp_mode`), bits:                 */
/*   OR_BP_CRC_STOP   stop when the CRC of the hard-decided u holds (Sec. II-B, the paper's rule) */
/*   OR_BP_REENC_STOP stop when the hard decision of LLR(x) equals the re-encoded hard decision  */
/*                    of LLR(u), x = u G (Sec. II-B, the stopping condition the CRC replaces)     */
/*   OR_BP_G_EXACT    the exact PE function g(a, b) = ln((1 + e^(a+b)) / (e^a + e^b)) instead of  */
/*                    the min-sum approximation (Sec. II-B)                                       */
#define OR_BP_CRC_STOP 1
#define OR_BP_REENC_STOP 2
#define OR_BP_G_EXACT 4

/* ------------------------------------------------------------------------------------------ */
/* Type-generic decoders: BP, SC, SCL, hybrid, in FP32 (bit-exact parity target), FP64 (FER ref.) */
/* and FP16-emulated (half-precision BP messages).                                           */
/* ------------------------------------------------------------------------------------------ */
#define OR_ROUND(x) (x)
#define REAL float
#define SFX(name) name##_f32
#include "polar_oracle_decoders.inc"
#undef REAL
#undef SFX

#define REAL double
#define SFX(name) name##_f64
#include "polar_oracle_decoders.inc"
#undef REAL
#undef SFX
#undef OR_ROUND

#define OR_ROUND(x) or_round_half(x)
#define OR_HALF_BP 1
#define REAL float
#define SFX(name) name##_f16
#include "polar_oracle_decoders.inc"
#undef REAL
#undef SFX
#undef OR_ROUND

/* ------------------------------------------------------------------------------------------ */
/* Brute-force ML over all 2^K information words (tiny codes only): the codeword minimising   */
/* the correlation discrepancy sum_j |lambda_j| [x_j != HD(lambda_j)].  Used only to pin SCL.  */
/* ------------------------------------------------------------------------------------------ */
double or_ml_decode(const double* llr, int N, int K, const int* info_idx, unsigned char* u_best)
{
    unsigned char* u = (unsigned char*)malloc((size_t)N);
    unsigned char* x = (unsigned char*)malloc((size_t)N);
    double best = INFINITY;
    for (long long w = 0; w < (1LL << K); ++w) {
        memset(u, 0, (size_t)N);
        for (int k = 0; k < K; ++k) u[info_idx[k]] = (unsigned char)((w >> (K - 1 - k)) & 1);
        or_polar_transform(u, N, x);
        double d = 0.0;
        for (int j = 0; j < N; ++j) {
            int hd = llr[j] < 0.0;
            if (x[j] != hd) d += fabs(llr[j]);
        }
        if (d < best) {
            best = d;
            memcpy(u_best, u, (size_t)N);
        }
    }
    free(u);
    free(x);
    return best;
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
