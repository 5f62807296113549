/*
 * Plain CPU oracle for the parallel block-based Viterbi decoder (PBVD).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; it is written from the paper's equations,
 * in the paper's notation, with 64-bit path metrics, no SIMD and no blocking
 * or reordering beyond what the method itself states.
 *
 * Paper: Peng, Liu, Hou, Zhao, "A Gb/s Parallel Block-based Viterbi Decoder
 * for Convolutional Codes on GPU" (arXiv 1608.00066).
 *
 * What each function follows:
 *   orc_codeword        Eq. (2): output of the (R,1,K) encoder for state S_d
 *                       and input bit x; state d = (D_{v-1} ... D_0)_2.
 *   orc_next_state      Sec. III-B butterfly: S_{2j}, S_{2j+1} -> S_j (x = 0)
 *                       or S_{j + 2^{v-1}} (x = 1).
 *   orc_encode          the encoder of Eq. (2) run as a shift register,
 *                       zero-terminated with v tail bits.
 *   orc_branch_metric   Sec. II: distance from the received soft values to a
 *                       codeword (Euclidean-style L1 distance on int8 LLRs).
 *   orc_acs_stage       Eq. (1) with the predecessor pair of the butterfly.
 *   orc_viterbi_full    Sec. II full-frame VA, known start state S_0,
 *                       traceback from S_0 at the last stage (terminated).
 *   orc_viterbi_block   Sec. III-A / Algorithm 1: blocks of D stages, L
 *                       truncation stages before and L traceback stages after,
 *                       zero initial metrics, traceback from S_0, no argmin.
 *   orc_brute_force     the maximum-likelihood definition the VA computes
 *                       (Sec. II): exhaustive search over all 2^k messages.
 *   orc_depuncture      puncturing is not in the paper; punctured positions
 *                       are read as erasures (LLR 0), which add the same
 *                       amount to every branch metric.
 *   orc_viterbi_block_variant  the block form with the argmin start state
 *                       of the classic VA (Sec. II) and/or circular windows
 *                       for tail-biting frames (not in the paper);
 *   orc_encode_tailbiting  tail-biting encoder (start state = end state);
 *   orc_unpack_soft, orc_branch_metric_q, orc_viterbi_block_q
 *                       Sec. IV-C: q-bit soft values packed floor(32/q) to a
 *                       32-bit word (q = 1: hard decisions), decoded by the
 *                       block form with mu = +-Q, Q = 2^{q-1} - 1;
 *   orc_viterbi_window  continuous (carried-metric) form for streaming:
 *                       Eq. (1) run without restarts over an unbounded stream;
 *                       each segment of D stages is released once L further
 *                       stages exist, by traceback from S_0 over those L.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - branch metric: BM(c) = sum_r |lambda_r - mu(c^(r))|, mu(0) = +127,
 *     mu(1) = -127, lambda = -128 read as -127;
 *   - ties in Eq. (1): the upper branch (predecessor S_{2j}, survivor bit 0)
 *     wins, i.e. the survivor bit is 1 only when the lower branch is strictly
 *     smaller;
 *   - known start: PM(S_0) = 0 and PM(other) = ORC_BIG = 8192;
 *   - first block: its truncation range is clamped at stage 0 and it starts
 *     from the known state S_0; last block: clamped at the last stage and
 *     traced back from S_0 (streams are zero-terminated).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BIG 8192
#define ORC_MAX_R 8
#define ORC_MAX_K 16

/* ---------------------------------------------------------------- code -- */

/* Eq. (2): c^(r) = (x*g^(r)_{K-1}) xor (D_{K-2}*g^(r)_{K-2}) xor ... xor (D_0*g^(r)_0).
 * Bit m of the integer g is g_m (the leftmost octal digit holds g_{K-1}). */
static int orc_filter_output(uint32_t g, int K, uint32_t d, int x)
{
    int c = x & (int)((g >> (K - 1)) & 1u);
    for (int m = 0; m <= K - 2; m++) {
        int D_m = (int)((d >> m) & 1u);
        int g_m = (int)((g >> m) & 1u);
        c ^= D_m & g_m;
    }
    return c;
}

/* c(S_d, x) = [c^(1) c^(2) ... c^(R)] packed with c^(1) as the most
 * significant bit, the order in which Table 2 prints alpha..theta. */
uint32_t orc_codeword(int K, int R, const uint32_t *gens, uint32_t d, int x)
{
    uint32_t c = 0;
    for (int r = 0; r < R; r++)
        c = (c << 1) | (uint32_t)orc_filter_output(gens[r], K, d, x);
    return c;
}

/* Butterfly of Sec. III-B: S_{2j} and S_{2j+1} move to S_j for x = 0 and to
 * S_{j+2^{v-1}} for x = 1, i.e. the new input bit becomes D_{v-1}. */
uint32_t orc_next_state(int K, uint32_t d, int x)
{
    int v = K - 1;
    return (d >> 1) | ((uint32_t)x << (v - 1));
}

/* Fills table[d*2 + x] = c(S_d, x) for all N = 2^{K-1} states. */
void orc_output_table(int K, int R, const uint32_t *gens, uint32_t *table)
{
    uint32_t N = 1u << (K - 1);
    for (uint32_t d = 0; d < N; d++)
        for (int x = 0; x < 2; x++)
            table[d * 2 + x] = orc_codeword(K, R, gens, d, x);
}

/* Zero-terminated encoding: k message bits followed by v zero tail bits,
 * n = k + v stages, R code bits per stage written stage-major into out. */
int64_t orc_encode(int K, int R, const uint32_t *gens, const uint8_t *msg,
                   int64_t k, uint8_t *out)
{
    int v = K - 1;
    uint32_t d = 0; /* encoder starts in S_0 */
    int64_t n = k + v;
    for (int64_t s = 0; s < n; s++) {
        int x = s < k ? (msg[s] & 1) : 0;
        uint32_t c = orc_codeword(K, R, gens, d, x);
        for (int r = 0; r < R; r++)
            out[s * R + r] = (uint8_t)((c >> (R - 1 - r)) & 1u);
        d = orc_next_state(K, d, x);
    }
    return n;
}

/* ----------------------------------------------------------- puncturing -- */

/* pattern is R x P row-major: code bit r of stage s is sent iff
 * pattern[r*P + s%P] != 0.  Sent values are stage-major, r ascending. */
int64_t orc_puncture(int R, const uint8_t *pattern, int P, const uint8_t *bits,
                     int64_t n, uint8_t *out)
{
    int64_t o = 0;
    for (int64_t s = 0; s < n; s++)
        for (int r = 0; r < R; r++)
            if (pattern[r * P + (int)(s % P)])
                out[o++] = bits[s * R + r];
    return o;
}

/* Inverse of orc_puncture on soft values: punctured positions become 0. */
int64_t orc_depuncture(int R, const uint8_t *pattern, int P, const int8_t *llr_tx,
                       int64_t n, int8_t *llr_full)
{
    int64_t i = 0;
    for (int64_t s = 0; s < n; s++)
        for (int r = 0; r < R; r++)
            llr_full[s * R + r] = pattern[r * P + (int)(s % P)] ? llr_tx[i++] : 0;
    return i;
}

/* ------------------------------------------------------------- metrics -- */

/* Distance from the received soft values of one stage to codeword c:
 * sum over r of |lambda_r - mu(c^(r))| with mu(0) = +127 and mu(1) = -127. */
int64_t orc_branch_metric(int R, const int8_t *lam, uint32_t c)
{
    int64_t bm = 0;
    for (int r = 0; r < R; r++) {
        int64_t l = lam[r] < -127 ? -127 : lam[r];
        int bit = (int)((c >> (R - 1 - r)) & 1u);
        int64_t mu = bit ? -127 : 127;
        int64_t diff = l - mu;
        bm += diff < 0 ? -diff : diff;
    }
    return bm;
}

/* Eq. (1) for one stage: PM_n^j = min_i (PM_{n-1}^i + BM_n^{i,j}) over the
 * two states i that reach j.  Those are S_{2j'} and S_{2j'+1} with
 * j' = j mod 2^{v-1}, taking input x = j >> (v-1).  dec[j] = 1 records that
 * the lower predecessor S_{2j'+1} was kept; a tie keeps the upper one. */
void orc_acs_stage(int K, int R, const uint32_t *gens, const int8_t *lam,
                   const int64_t *pm_prev, int64_t *pm_next, uint8_t *dec)
{
    int v = K - 1;
    uint32_t N = 1u << v;
    for (uint32_t j = 0; j < N; j++) {
        uint32_t jp = j & ((1u << (v - 1)) - 1u);
        int x = (int)(j >> (v - 1));
        uint32_t i0 = 2 * jp, i1 = 2 * jp + 1;
        int64_t m0 = pm_prev[i0] + orc_branch_metric(R, lam, orc_codeword(K, R, gens, i0, x));
        int64_t m1 = pm_prev[i1] + orc_branch_metric(R, lam, orc_codeword(K, R, gens, i1, x));
        if (m1 < m0) {
            pm_next[j] = m1;
            dec[j] = 1;
        } else {
            pm_next[j] = m0;
            dec[j] = 0;
        }
    }
}

/* Predecessor on the survivor path (Algorithm 1, backward procedure):
 * state = 2 * (state mod 2^{v-1}) + sp. */
static uint32_t orc_predecessor(int K, uint32_t state, int sp)
{
    int v = K - 1;
    return 2u * (state & ((1u << (v - 1)) - 1u)) + (uint32_t)sp;
}

/* Decoded bit of a state: its most significant memory cell D_{v-1}, which
 * holds the input bit that led into it (Algorithm 1: (state >> (K-2)) & 1). */
static int orc_state_bit(int K, uint32_t state)
{
    return (int)((state >> (K - 2)) & 1u);
}

/* --------------------------------------------------------- full frame -- */

/* Full-frame VA over n stages of mother-code soft values (n*R int8, stage
 * major).  Starts in the known state S_0, traces back from S_0 at stage n-1.
 * out[s] = decoded bit of stage s (one per byte).  Optional outputs: the final
 * metrics (N values), every survivor bit dec[s*N + j] and every metric
 * pm_trace[s*N + j] after stage s.  Returns 0, or -1 on allocation failure. */
int orc_viterbi_full(int K, int R, const uint32_t *gens, const int8_t *llr, int64_t n,
                     uint8_t *out, int64_t *final_pm, uint8_t *dec_out, int64_t *pm_trace)
{
    int v = K - 1;
    uint32_t N = 1u << v;
    if (n <= 0)
        return 0;
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *pm2 = (int64_t *)malloc(sizeof(int64_t) * N);
    uint8_t *dec = (uint8_t *)malloc((size_t)n * N);
    if (!pm || !pm2 || !dec) {
        free(pm); free(pm2); free(dec);
        return -1;
    }
    for (uint32_t j = 0; j < N; j++)
        pm[j] = j == 0 ? 0 : ORC_BIG;
    for (int64_t s = 0; s < n; s++) {
        orc_acs_stage(K, R, gens, llr + s * R, pm, pm2, dec + s * N);
        int64_t *t = pm; pm = pm2; pm2 = t;
        if (pm_trace)
            memcpy(pm_trace + s * N, pm, sizeof(int64_t) * N);
    }
    if (final_pm)
        memcpy(final_pm, pm, sizeof(int64_t) * N);
    uint32_t state = 0;
    for (int64_t s = n - 1; s >= 0; s--) {
        out[s] = (uint8_t)orc_state_bit(K, state);
        state = orc_predecessor(K, state, dec[s * N + state]);
    }
    if (dec_out)
        memcpy(dec_out, dec, (size_t)n * N);
    free(pm); free(pm2); free(dec);
    return 0;
}

/* -------------------------------------------------------- block-based -- */

/* Geometry of parallel block b (Sec. III-A, Fig. 1): it decodes stages
 * [bD, min((b+1)D, n)); its forward range runs from f0 = max(0, bD - L)
 * to f1 = min(n, (b+1)D + L) - 1. */
void orc_block_geometry(int64_t n, int64_t D, int64_t L, int64_t b,
                        int64_t *f0, int64_t *f1, int64_t *o0, int64_t *o1)
{
    int64_t s = b * D - L;
    int64_t e = (b + 1) * D + L;
    *f0 = s < 0 ? 0 : s;
    *f1 = (e < n ? e : n) - 1;
    *o0 = b * D;
    *o1 = (b + 1) * D < n ? (b + 1) * D : n;
}

/* Decodes blocks b in [b_begin, b_end) of a stream of n stages, each on its
 * own: fresh metrics (known start if the block's range begins at stage 0,
 * all zero otherwise), Eq. (1) over [f0, f1], traceback from S_0 at f1 with
 * no metric comparison, and output of the stages [bD, min((b+1)D, n)).
 * out is indexed by absolute stage.  When pm_end is not NULL,
 * pm_end[b - b_begin] receives PM(S_0) after stage f1: the metric of the path
 * the traceback follows.  Returns 0, or -1 on bad arguments or allocation
 * failure. */
int orc_viterbi_block_metrics(int K, int R, const uint32_t *gens, const int8_t *llr, int64_t n,
                              int64_t D, int64_t L, int64_t b_begin, int64_t b_end, uint8_t *out,
                              int64_t *pm_end)
{
    int v = K - 1;
    uint32_t N = 1u << v;
    if (D <= 0 || L < 0)
        return -1;
    if (n <= 0)
        return 0;
    int64_t span = D + 2 * L;
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *pm2 = (int64_t *)malloc(sizeof(int64_t) * N);
    uint8_t *dec = (uint8_t *)malloc((size_t)span * N);
    if (!pm || !pm2 || !dec) {
        free(pm); free(pm2); free(dec);
        return -1;
    }
    for (int64_t b = b_begin; b < b_end; b++) {
        int64_t f0, f1, o0, o1;
        orc_block_geometry(n, D, L, b, &f0, &f1, &o0, &o1);
        for (uint32_t j = 0; j < N; j++)
            pm[j] = (f0 == 0) ? (j == 0 ? 0 : ORC_BIG) : 0;
        for (int64_t s = f0; s <= f1; s++) {
            orc_acs_stage(K, R, gens, llr + s * R, pm, pm2, dec + (s - f0) * N);
            int64_t *t = pm; pm = pm2; pm2 = t;
        }
        if (pm_end)
            pm_end[b - b_begin] = pm[0];
        uint32_t state = 0;
        for (int64_t s = f1; s >= o0; s--) {
            if (s < o1)
                out[s] = (uint8_t)orc_state_bit(K, state);
            state = orc_predecessor(K, state, dec[(s - f0) * N + state]);
        }
    }
    free(pm); free(pm2); free(dec);
    return 0;
}

int orc_viterbi_block_range(int K, int R, const uint32_t *gens, const int8_t *llr, int64_t n,
                            int64_t D, int64_t L, int64_t b_begin, int64_t b_end, uint8_t *out)
{
    return orc_viterbi_block_metrics(K, R, gens, llr, n, D, L, b_begin, b_end, out, NULL);
}

/* Variants of the block form (Sec. III-A) selected by flags:
 *   ORC_TB_ARGMIN  the traceback of every block starts from the state with
 *                  the smallest metric at f1 (the start state S_E of the
 *                  classic VA, Sec. II), the lowest state index on ties,
 *                  instead of S_0;
 *   ORC_CIRCULAR   tail-biting frames (not in the paper): the frame is a
 *                  circle of n stages, stage s reads the soft values of stage
 *                  s mod n; block b's window is [o0 - L, o1 + L - 1] with no
 *                  clamping and every block starts from zero metrics (the
 *                  encoder's start state is unknown).
 * With flags = 0 this is orc_viterbi_block_metrics.  pm_end (optional)
 * receives the metric of the traceback's start state per block. */
#define ORC_TB_ARGMIN 1
#define ORC_CIRCULAR 2

int orc_viterbi_block_variant(int K, int R, const uint32_t *gens, const int8_t *llr, int64_t n,
                              int64_t D, int64_t L, int64_t b_begin, int64_t b_end, int flags,
                              uint8_t *out, int64_t *pm_end)
{
    int v = K - 1;
    uint32_t N = 1u << v;
    int circular = (flags & ORC_CIRCULAR) != 0;
    if (D <= 0 || L < 0)
        return -1;
    if (n <= 0)
        return 0;
    int64_t span = D + 2 * L;
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *pm2 = (int64_t *)malloc(sizeof(int64_t) * N);
    uint8_t *dec = (uint8_t *)malloc((size_t)span * N);
    if (!pm || !pm2 || !dec) {
        free(pm); free(pm2); free(dec);
        return -1;
    }
    for (int64_t b = b_begin; b < b_end; b++) {
        int64_t f0, f1, o0, o1;
        orc_block_geometry(n, D, L, b, &f0, &f1, &o0, &o1);
        if (circular) {
            f0 = o0 - L;
            f1 = o1 + L - 1;
        }
        int known = !circular && f0 == 0;
        for (uint32_t j = 0; j < N; j++)
            pm[j] = known ? (j == 0 ? 0 : ORC_BIG) : 0;
        for (int64_t s = f0; s <= f1; s++) {
            int64_t sm = ((s % n) + n) % n;
            orc_acs_stage(K, R, gens, llr + sm * R, pm, pm2, dec + (s - f0) * N);
            int64_t *t = pm; pm = pm2; pm2 = t;
        }
        uint32_t state = 0;
        if (flags & ORC_TB_ARGMIN) {
            for (uint32_t j = 1; j < N; j++)
                if (pm[j] < pm[state])
                    state = j;
        }
        if (pm_end)
            pm_end[b - b_begin] = pm[state];
        for (int64_t s = f1; s >= o0; s--) {
            if (s < o1)
                out[s] = (uint8_t)orc_state_bit(K, state);
            state = orc_predecessor(K, state, dec[(s - f0) * N + state]);
        }
    }
    free(pm); free(pm2); free(dec);
    return 0;
}

/* Tail-biting encoding (not in the paper): the encoder starts in the state
 * its last v message bits leave it in, so that it ends where it started; k
 * stages, no tail.  Needs k >= v.  out as for orc_encode. */
int64_t orc_encode_tailbiting(int K, int R, const uint32_t *gens, const uint8_t *msg, int64_t k,
                              uint8_t *out)
{
    int v = K - 1;
    if (k < v)
        return -1;
    uint32_t d = 0;
    for (int64_t s = k - v; s < k; s++)
        d = orc_next_state(K, d, msg[s] & 1);
    for (int64_t s = 0; s < k; s++) {
        int x = msg[s] & 1;
        uint32_t c = orc_codeword(K, R, gens, d, x);
        for (int r = 0; r < R; r++)
            out[s * R + r] = (uint8_t)((c >> (R - 1 - r)) & 1u);
        d = orc_next_state(K, d, x);
    }
    return k;
}

int orc_viterbi_block(int K, int R, const uint32_t *gens, const int8_t *llr, int64_t n,
                      int64_t D, int64_t L, uint8_t *out)
{
    if (D <= 0)
        return -1;
    int64_t nb = (n + D - 1) / D;
    return orc_viterbi_block_range(K, R, gens, llr, n, D, L, 0, nb, out);
}

/* ------------------------------------------- q-bit quantised inputs -- */

/* Sec. IV-C: soft values quantised to q bits, floor(32/q) of them packed in
 * one 32-bit word: value i sits in word i / m (m = floor(32/q)) at bits
 * [q (i mod m), q (i mod m) + q), as a q-bit two's complement number.  q = 1
 * is hard decision: the bit is the received code bit, read as +1 (bit 0) or
 * -1 (bit 1).  Unpacks count values into out.  Returns 0, -1 for bad q. */
int orc_unpack_soft(int q, const uint32_t *words, int64_t count, int8_t *out)
{
    if (q < 1 || q > 8)
        return -1;
    int64_t m = 32 / q;
    for (int64_t i = 0; i < count; i++) {
        uint32_t w = words[i / m];
        int shift = (int)(q * (i % m));
        uint32_t u = (w >> shift) & ((1u << q) - 1u);
        if (q == 1) {
            out[i] = u ? -1 : 1;
        } else {
            int32_t val = (int32_t)u;
            if (u & (1u << (q - 1)))
                val -= (int32_t)(1u << q);
            out[i] = (int8_t)val;
        }
    }
    return 0;
}

/* The branch metric of Sec. II on q-bit values: sum_r |lambda_r - mu(c_r)|
 * with mu(0) = +Q, mu(1) = -Q, Q = 2^{q-1} - 1 the largest magnitude (Q = 1
 * for hard decisions, where the metric is twice the Hamming distance);
 * values below -Q read as -Q. */
int64_t orc_branch_metric_q(int R, const int8_t *lam, uint32_t c, int Q)
{
    int64_t bm = 0;
    for (int r = 0; r < R; r++) {
        int64_t l = lam[r] < -Q ? -Q : lam[r];
        int bit = (int)((c >> (R - 1 - r)) & 1u);
        int64_t mu = bit ? -Q : Q;
        int64_t diff = l - mu;
        bm += diff < 0 ? -diff : diff;
    }
    return bm;
}

/* Eq. (1) for one stage with orc_branch_metric_q (tie rule as orc_acs_stage). */
void orc_acs_stage_q(int K, int R, const uint32_t *gens, const int8_t *lam, int Q,
                     const int64_t *pm_prev, int64_t *pm_next, uint8_t *dec)
{
    int v = K - 1;
    uint32_t N = 1u << v;
    for (uint32_t j = 0; j < N; j++) {
        uint32_t jp = j & ((1u << (v - 1)) - 1u);
        int x = (int)(j >> (v - 1));
        uint32_t i0 = 2 * jp, i1 = 2 * jp + 1;
        int64_t m0 = pm_prev[i0] + orc_branch_metric_q(R, lam, orc_codeword(K, R, gens, i0, x), Q);
        int64_t m1 = pm_prev[i1] + orc_branch_metric_q(R, lam, orc_codeword(K, R, gens, i1, x), Q);
        if (m1 < m0) {
            pm_next[j] = m1;
            dec[j] = 1;
        } else {
            pm_next[j] = m0;
            dec[j] = 0;
        }
    }
}

/* The block form (Sec. III-A, Algorithm 1) on unpacked q-bit values
 * (n * R of them, stage major) with the metric of orc_branch_metric_q. */
int orc_viterbi_block_q(int K, int R, const uint32_t *gens, const int8_t *llr_q, int64_t n,
                        int64_t D, int64_t L, int Q, uint8_t *out)
{
    int v = K - 1;
    uint32_t N = 1u << v;
    if (D <= 0 || L < 0 || Q < 1)
        return -1;
    if (n <= 0)
        return 0;
    int64_t span = D + 2 * L;
    int64_t nb = (n + D - 1) / D;
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *pm2 = (int64_t *)malloc(sizeof(int64_t) * N);
    uint8_t *dec = (uint8_t *)malloc((size_t)span * N);
    if (!pm || !pm2 || !dec) {
        free(pm); free(pm2); free(dec);
        return -1;
    }
    for (int64_t b = 0; b < nb; b++) {
        int64_t f0, f1, o0, o1;
        orc_block_geometry(n, D, L, b, &f0, &f1, &o0, &o1);
        for (uint32_t j = 0; j < N; j++)
            pm[j] = (f0 == 0) ? (j == 0 ? 0 : ORC_BIG) : 0;
        for (int64_t s = f0; s <= f1; s++) {
            orc_acs_stage_q(K, R, gens, llr_q + s * R, Q, pm, pm2, dec + (s - f0) * N);
            int64_t *t = pm; pm = pm2; pm2 = t;
        }
        uint32_t state = 0;
        for (int64_t s = f1; s >= o0; s--) {
            if (s < o1)
                out[s] = (uint8_t)orc_state_bit(K, state);
            state = orc_predecessor(K, state, dec[(s - f0) * N + state]);
        }
    }
    free(pm); free(pm2); free(dec);
    return 0;
}

/* ----------------------------------------------- carried-metric stream -- */

/* Continuous form for streams fed in pieces: Eq. (1) is run once over the
 * whole stream with metrics carried from stage to stage (known start S_0).
 * Segment m = [mD, (m+1)D) is released when stage (m+1)D + L - 1 exists, by
 * traceback from S_0 at that stage; the final partial segment is released
 * at the end of the (zero-terminated) stream by traceback from S_0 at the last
 * stage.  Memory grows with n; this is a definition, not an implementation. */
int orc_viterbi_window(int K, int R, const uint32_t *gens, const int8_t *llr, int64_t n,
                       int64_t D, int64_t L, uint8_t *out)
{
    int v = K - 1;
    uint32_t N = 1u << v;
    if (D <= 0 || L < 0)
        return -1;
    if (n <= 0)
        return 0;
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *pm2 = (int64_t *)malloc(sizeof(int64_t) * N);
    uint8_t *dec = (uint8_t *)malloc((size_t)n * N);
    if (!pm || !pm2 || !dec) {
        free(pm); free(pm2); free(dec);
        return -1;
    }
    for (uint32_t j = 0; j < N; j++)
        pm[j] = j == 0 ? 0 : ORC_BIG;
    int64_t released = 0; /* first stage not yet decoded */
    for (int64_t s = 0; s < n; s++) {
        orc_acs_stage(K, R, gens, llr + s * R, pm, pm2, dec + s * N);
        int64_t *t = pm; pm = pm2; pm2 = t;
        int64_t seg_end = released + D;
        int last = (s == n - 1);
        if (last || s == seg_end + L - 1) {
            int64_t o1 = last ? n : seg_end;
            uint32_t state = 0;
            for (int64_t q = s; q >= released; q--) {
                if (q < o1)
                    out[q] = (uint8_t)orc_state_bit(K, state);
                state = orc_predecessor(K, state, dec[q * N + state]);
            }
            released = o1;
            /* a terminated stream may still hold full segments after the
             * last traceback above; they were all written by it */
        }
    }
    free(pm); free(pm2); free(dec);
    return 0;
}

/* --------------------------------------------------------- brute force -- */

/* Maximum-likelihood search over all 2^k messages (k <= 24), each encoded
 * with v zero tail bits: the sum of branch metrics along the codeword.  Gives
 * the smallest metric, the first message (in increasing integer order, bit s
 * of the integer = message bit s) that reaches it and how many do. */
int orc_brute_force(int K, int R, const uint32_t *gens, const int8_t *llr, int k,
                    uint8_t *best_msg, int64_t *best_metric, int64_t *n_best)
{
    int v = K - 1;
    if (k < 0 || k > 24)
        return -1;
    int64_t n = (int64_t)k + v;
    int64_t best = -1, count = 0;
    uint64_t best_m = 0;
    for (uint64_t m = 0; m < (1ull << k); m++) {
        uint32_t d = 0;
        int64_t metric = 0;
        for (int64_t s = 0; s < n; s++) {
            int x = s < k ? (int)((m >> s) & 1u) : 0;
            metric += orc_branch_metric(R, llr + s * R, orc_codeword(K, R, gens, d, x));
            d = orc_next_state(K, d, x);
        }
        if (best < 0 || metric < best) {
            best = metric;
            best_m = m;
            count = 1;
        } else if (metric == best) {
            count++;
        }
    }
    for (int s = 0; s < k; s++)
        best_msg[s] = (uint8_t)((best_m >> s) & 1u);
    *best_metric = best;
    *n_best = count;
    return 0;
}
