/*
 * ppf_oracle.c -- plain, slow FP64 CPU reference of the SIR time step of
 * "PPF - A Parallel Particle Filtering Library" (Demirel et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or constant generator with the CUDA library; both sides
 * implement the same published definitions independently.
 *
 * What it follows, step by step (Alg. 1, Sec. 2):
 *   init        Alg. 1 initialisation: w = 1/N, x_0 drawn from a uniform
 *               prior over the image (Sec. 7.3).
 *   propagate   Alg. 1 SIS draw with the bootstrap proposal pi = p(x_k|x_{k-1}),
 *               the near-constant-velocity model of Sec. 7.1.
 *   weight      Alg. 1 weight update, likelihood eq. 4 with the appearance
 *               model eq. 3 over the (2r+1)^2 patch S_x.
 *   summary     Alg. 1 normalisation and effective sample size, the MMSE
 *               estimate of Sec. 2, and the per-frame log-evidence.
 *   quantise /  Alg. 1 resampling step (Pr[s(i)=l] = w_l), realised as
 *   systematic  systematic resampling on 64-bit fixed-point weights.
 *   schedule    Sec. 4: Greedy (Alg. 2), Sorted Greedy (Alg. 3) and Largest
 *               Gradient (Alg. 4) schedulers for RPA particle routing.
 *   resample    Sec. 3: RPA (proportional allocation, one- and two-stage)
 *               and RNA (local resampling + ring migration); Sec. 7's ARNA
 *               (adaptive exchange ratio, ring redrawn when the object is
 *               lost).
 *
 * Readings of points the paper leaves open (kept identical on the CUDA side):
 *   - dynamics (Sec. 7.1 names the model, gives no equations):
 *       x' = x + vx + sm*e1, y' = y + vy + sm*e2, vx' = vx + sv*e3,
 *       vy' = vy + sv*e4, I0' = I0 + sI*e5, one frame per step.
 *   - patch S_x: a fixed (2r+1)x(2r+1) box centred on c = floor(x + 1/2);
 *     pixels outside the image are left out of the sum.  Pixels outside S_x
 *     are modelled as background, so the factor that eq. 4's proportionality
 *     leaves out is the particle-independent whole-frame background term:
 *       l = -sum_{S_x} [(Z - I)^2 - (Z - I_bg)^2] / (2 sigma_xi^2).
 *     (For particles sharing an anchor this equals the literal form up to a
 *     constant; across anchors it keeps particles that leave the image from
 *     winning with an empty sum.)
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *     key = (seed_lo, seed_hi), counter = (index, frame, filter, purpose<<8|block);
 *     prior uniforms u = (2*(r>>9)+1) * 2^-24 from 32-bit words; propagation
 *     uniforms from six 21-bit fields of one block, u = (2 f + 1) 2^-22 (both
 *     exact in float32); Box-Muller normals.
 *   - resampling weights: q_i = floor(2^(s + t_i)) with t_i = (lw_i - M) log2 e,
 *     evaluated in float32 by a fixed operation sequence (a float decides an
 *     integer here, so the oracle takes that decision in the kernel's float32
 *     precision), s = 63 - ceil(log2 n); ticket offset u = floor(r64 * Q / 2^64).
 *
 * parity pins: every function here is checked by the CPU test-suite against a
 * closed form, a library routine, an invariant or brute force.  Two readings
 * are parity unpinned, as the papers that define them are not available:
 * that the piecewise constant likelihood below (likelihood = 1) is the cited
 * pcSIR, and that orc_resample_arna's rules (involved groups, ratio, loss
 * test, ring order) are the cited ARNA.  The functions themselves are pinned
 * (constant cells and centre value; ring order against Philox, the exchange
 * against RNA's local draws and the involved count against the systematic
 * draw).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "ppf_oracle.h"

/* Threads: the per-particle loops (init, propagation, likelihood, the
 * exponentials of the summary) may run in parallel over particles; each
 * particle's arithmetic is unchanged and every reduction is summed serially
 * in particle order, so results do not depend on the thread count. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11: "Parallel random numbers: as easy as  */
/* 1, 2, 3").  Round: two 32x32->64 products of counter words 0 and 2 with    */
/* the multipliers, xor of the high halves with the other counter words and  */
/* the key; the key is bumped by the Weyl constants between rounds.           */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t index, uint32_t frame, uint32_t filter,
                 uint32_t purpose, uint32_t block, uint32_t out[4])
{
    uint32_t ctr[4] = {index, frame, filter, (purpose << 8) | block};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

double orc_u01(uint32_t r)
{
    /* odd multiple of 2^-24 in (0, 1): exactly representable in float32 */
    return (double)(2u * (r >> 9) + 1u) * (1.0 / 16777216.0);
}

/* The propagation noise of one slot comes from one Philox block: its 128 bits
 * (word 0 least significant) are cut into six 21-bit fields, field k holding
 * bits [21k, 21k + 21); each becomes u = (2 field + 1) 2^-22 (exact in float32)
 * and the three Box-Muller pairs (u0,u1), (u2,u3), (u4,u5) give the normals. */
double orc_u21(uint32_t field)
{
    return (double)(2u * (field & 0x1FFFFFu) + 1u) * (1.0 / 4194304.0);
}

void orc_prop_fields(const uint32_t r[4], uint32_t f[6])
{
    unsigned __int128 b = (unsigned __int128)r[0] | ((unsigned __int128)r[1] << 32) |
                          ((unsigned __int128)r[2] << 64) | ((unsigned __int128)r[3] << 96);
    for (int k = 0; k < 6; ++k)
        f[k] = (uint32_t)((b >> (21 * k)) & 0x1FFFFFu);
}

static void box_muller_u(double u1, double u2, double *z0, double *z1)
{
    const double two_pi = 6.283185307179586476925286766559;
    double rho = sqrt(-2.0 * log(u1));
    *z0 = rho * cos(two_pi * u2);
    *z1 = rho * sin(two_pi * u2);
}

void orc_normals5(uint64_t seed, uint32_t slot, uint32_t frame, uint32_t filter, double e[5])
{
    uint32_t r[4], f[6];
    draw(seed, slot, frame, filter, ORC_PURPOSE_PROP, 0, r);
    orc_prop_fields(r, f);
    double spare;
    box_muller_u(orc_u21(f[0]), orc_u21(f[1]), &e[0], &e[1]);
    box_muller_u(orc_u21(f[2]), orc_u21(f[3]), &e[2], &e[3]);
    box_muller_u(orc_u21(f[4]), orc_u21(f[5]), &e[4], &spare);
}

/* ------------------------------------------------------------------------ */
/* S0: initialisation (Alg. 1, k = 0; particles drawn uniformly, Sec. 7.3)   */
/* ------------------------------------------------------------------------ */
void orc_init(const orc_model *m, int64_t N, double *st)
{
    double *x = st, *y = st + N, *vx = st + 2 * N, *vy = st + 3 * N, *I0 = st + 4 * N, *lw = st + 5 * N;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        uint32_t a[4], b[4];
        draw(m->seed, (uint32_t)i, 0u, m->filter_id, ORC_PURPOSE_INIT, 0, a);
        draw(m->seed, (uint32_t)i, 0u, m->filter_id, ORC_PURPOSE_INIT, 1, b);
        x[i] = -0.5 + (double)m->width * orc_u01(a[0]);
        y[i] = -0.5 + (double)m->height * orc_u01(a[1]);
        vx[i] = m->v0_max * (2.0 * orc_u01(a[2]) - 1.0);
        vy[i] = m->v0_max * (2.0 * orc_u01(a[3]) - 1.0);
        I0[i] = m->amplitude * (0.5 + orc_u01(b[0]));
        lw[i] = 0.0; /* w_0 = 1/N: equal unnormalised log-weights */
    }
}

/* ------------------------------------------------------------------------ */
/* S1: bootstrap SIS draw (Alg. 1) with the NCV dynamics (Sec. 7.1).        */
/* Slot i takes parent anc[i]; its noise is keyed by (slot, frame).          */
/* The new log-weight starts at lw_prev[i] (the post-resampling weight).     */
/* ------------------------------------------------------------------------ */
void orc_propagate(const orc_model *m, int64_t N, int32_t frame, const double *par,
                   const int32_t *anc, const double *lw_prev, double *st)
{
    const double *px = par, *py = par + N, *pvx = par + 2 * N, *pvy = par + 3 * N, *pI = par + 4 * N;
    double *x = st, *y = st + N, *vx = st + 2 * N, *vy = st + 3 * N, *I0 = st + 4 * N, *lw = st + 5 * N;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t a = anc[i];
        double e[5];
        orc_normals5(m->seed, (uint32_t)i, (uint32_t)frame, m->filter_id, e);
        x[i] = px[a] + pvx[a] + m->sigma_m * e[0];
        y[i] = py[a] + pvy[a] + m->sigma_m * e[1];
        vx[i] = pvx[a] + m->sigma_v * e[2];
        vy[i] = pvy[a] + m->sigma_v * e[3];
        I0[i] = pI[a] + m->sigma_I * e[4];
        lw[i] = lw_prev[i];
    }
}

/* S1 for a sample of slots: parents5 holds, for each sampled slot, its parent's
 * (x, y, vx, vy, I0) as a 5 x n SoA; the noise is keyed by the slot index. */
void orc_propagate_slots(const orc_model *m, int64_t n, int32_t frame, const int64_t *slots,
                         const double *parents5, double *out5)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double e[5];
        orc_normals5(m->seed, (uint32_t)slots[k], (uint32_t)frame, m->filter_id, e);
        const double x = parents5[k], y = parents5[n + k], vx = parents5[2 * n + k];
        const double vy = parents5[3 * n + k], I0 = parents5[4 * n + k];
        out5[k] = x + vx + m->sigma_m * e[0];
        out5[n + k] = y + vy + m->sigma_m * e[1];
        out5[2 * n + k] = vx + m->sigma_v * e[2];
        out5[3 * n + k] = vy + m->sigma_v * e[3];
        out5[4 * n + k] = I0 + m->sigma_I * e[4];
    }
}

/* S3 for many particles: l[k] = loglik(x[k], y[k], I0[k]) */
void orc_loglik_many(const orc_model *m, const double *frame, int64_t n, const double *x, const double *y,
                     const double *I0, double *l)
{
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t k = 0; k < n; ++k)
        l[k] = orc_loglik(m, frame, x[k], y[k], I0[k]);
}

/* ------------------------------------------------------------------------ */
/* S3: log-likelihood of one particle, eq. 4 with the appearance model eq. 3 */
/* I(p) = I0 exp(-|p - (x,y)|^2 / (2 sigma^2)) + I_bg over the (2r+1)^2      */
/* pixels around c = floor((x,y) + 1/2) that lie inside the image.  Outside  */
/* S_x the frame is modelled as background, so eq. 4's proportionality holds */
/* for a window that moves with the particle: the particle-independent sum   */
/* of (Z - I_bg)^2 over the whole frame is dropped, leaving                  */
/*   l = -sum_{S_x} [(Z - I)^2 - (Z - I_bg)^2] / (2 sigma_xi^2).             */
/* frame: row-major H x W, values given as doubles (any storage precision   */
/* is converted by the caller).                                              */
/* ------------------------------------------------------------------------ */
double orc_loglik(const orc_model *m, const double *frame, double x, double y, double I0)
{
    if (!isfinite(x) || !isfinite(y) || !isfinite(I0))
        return -INFINITY;
    if (m->likelihood == 1) {
        /* pcSIR (Sec. 6): the likelihood is held constant on every pixel
         * cell [c - 1/2, c + 1/2)^2, at its value for the particle moved to
         * the cell centre c = floor((x, y) + 1/2) */
        x = floor(x + 0.5);
        y = floor(y + 0.5);
    }
    const int r = m->patch_radius;
    const double cxd = floor(x + 0.5), cyd = floor(y + 0.5);
    /* anchors far outside the image see no pixel: empty sum */
    if (cxd < -r - 1.0 || cxd > m->width + r || cyd < -r - 1.0 || cyd > m->height + r)
        return 0.0;
    const int64_t cx = (int64_t)cxd, cy = (int64_t)cyd;
    const double two_s2 = 2.0 * m->psf_sigma * m->psf_sigma;
    double sum = 0.0;
    for (int64_t py = cy - r; py <= cy + r; ++py) {
        if (py < 0 || py >= m->height)
            continue;
        for (int64_t px = cx - r; px <= cx + r; ++px) {
            if (px < 0 || px >= m->width)
                continue;
            double d2 = ((double)px - x) * ((double)px - x) + ((double)py - y) * ((double)py - y);
            double model = I0 * exp(-d2 / two_s2) + m->background;
            double z = frame[py * (int64_t)m->width + px];
            double res = z - model;          /* spot hypothesis, eq. 3 */
            double res0 = z - m->background; /* background-only hypothesis */
            sum += res * res - res0 * res0;
        }
    }
    return -sum / (2.0 * m->sigma_xi * m->sigma_xi);
}

void orc_weight(const orc_model *m, int64_t N, const double *frame, double *st)
{
    const double *x = st, *y = st + N, *I0 = st + 4 * N;
    double *lw = st + 5 * N;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < N; ++i)
        lw[i] += orc_loglik(m, frame, x[i], y[i], I0[i]);
}

/* ------------------------------------------------------------------------ */
/* S4/S5: normalisation, N_eff, MMSE estimate, log-evidence (Alg. 1, Sec. 2) */
/* out: mean[5], log_evidence, ess, max_lw                                    */
/* log-evidence = log sum_i e^{lw_i} - log sum_i e^{lw_prev_i}               */
/* ------------------------------------------------------------------------ */
void orc_summary(int64_t N, const double *st, const double *lw_prev, double out[8])
{
    /* a particle whose log-weight is -inf or NaN has zero weight: it is not
     * part of the weighted-sample approximation and adds nothing to any sum */
    const double *lw = st + 5 * N;
    double M = -INFINITY, Mp = -INFINITY;
    for (int64_t i = 0; i < N; ++i) {
        if (lw[i] > M) M = lw[i];
        if (lw_prev[i] > Mp) Mp = lw_prev[i];
    }
    /* the exponentials in parallel, the sums serially in particle order */
    double *e = (double *)malloc(sizeof(double) * (size_t)(2 * (N > 0 ? N : 1)));
    double *ep = e + N;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        e[i] = lw[i] > -INFINITY ? exp(lw[i] - M) : 0.0;
        ep[i] = lw_prev[i] > -INFINITY ? exp(lw_prev[i] - Mp) : 0.0;
    }
    double total = 0.0, totalp = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (lw[i] > -INFINITY)
            total += e[i];
        if (lw_prev[i] > -INFINITY)
            totalp += ep[i];
    }
    double mean[5] = {0, 0, 0, 0, 0}, sumsq = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (!(lw[i] > -INFINITY))
            continue;
        double w = e[i] / total;
        if (w == 0.0)
            continue;
        for (int c = 0; c < 5; ++c)
            mean[c] += w * st[c * N + i];
        sumsq += w * w;
    }
    free(e);
    for (int c = 0; c < 5; ++c)
        out[c] = mean[c];
    out[5] = (M + log(total)) - (Mp + log(totalp));
    out[6] = 1.0 / sumsq;
    out[7] = M;
}

/* ------------------------------------------------------------------------ */
/* S6: fixed-point resampling weight of one particle.                        */
/* q = floor(p * 2^(s+k)), t = (lw - M) * log2(e) in float32, k = floor(t),   */
/* f = t - k, p ~ 2^f by the degree-9 Taylor polynomial of e^(f ln 2)         */
/* (coefficients (ln 2)^n / n! rounded to float32), Horner with fused         */
/* multiply-add, all in float32.                                              */
/* ------------------------------------------------------------------------ */
int orc_scale_bits(int64_t n)
{
    int c = 0;
    while (((int64_t)1 << c) < n)
        ++c;
    return 63 - c;
}

float orc_exp2_frac(float f)
{
    /* (ln 2)^n / n!, n = 0..9, each rounded to the nearest float32 */
    static const float c[10] = {
        0x1p+0f,            0x1.62e43p-1f,     0x1.ebfbep-3f,     0x1.c6b08ep-5f,
        0x1.3b2ab6p-7f,     0x1.5d87fep-10f,   0x1.430912p-13f,   0x1.ffcbfcp-17f,
        0x1.62c022p-20f,    0x1.b5253ep-24f,
    };
    float p = c[9];
    for (int n = 8; n >= 0; --n)
        p = fmaf(p, f, c[n]);
    return p;
}

uint64_t orc_quantise(float lw, float M, int s)
{
    const float log2e = 0x1.715476p+0f; /* log2(e) rounded to float32 */
    float d = lw - M;
    float t = d * log2e;
    if (!(t > -64.0f))      /* also catches NaN */
        return 0;
    float kf = floorf(t);
    float f = t - kf;
    float p = orc_exp2_frac(f);
    int e = s + (int)kf;
    /* p in [1, 2]: P = p * 2^23 is an exact integer */
    uint64_t P = (uint64_t)ldexp((double)p, 23);
    if (e < -25)
        return 0;
    if (e >= 23)
        return P << (e - 23);
    return P >> (23 - e);
}

/* ------------------------------------------------------------------------ */
/* S7: systematic resampling on integers.                                    */
/* With inclusive sums C_i of q and total Q, ticket j (0 <= j < n) sits at    */
/* (u + j Q) / n and belongs to the first i with n * C_i > u + j Q.           */
/* T(c) = #{j : u + jQ < n c} = clamp(ceil((n c - u) / Q), 0, n).             */
/* ------------------------------------------------------------------------ */
typedef unsigned __int128 u128;

int64_t orc_tickets_below(uint64_t c, int64_t n, uint64_t u, uint64_t Q)
{
    u128 nc = (u128)c * (u128)(uint64_t)n;
    if (nc <= (u128)u)
        return 0;
    u128 num = nc - (u128)u;
    u128 t = (num + (u128)Q - 1) / (u128)Q;
    if (t > (u128)(uint64_t)n)
        t = (u128)(uint64_t)n;
    return (int64_t)t;
}

uint64_t orc_ticket_offset(uint64_t seed, uint32_t filter, uint32_t frame, uint32_t purpose,
                           uint32_t index, uint64_t Q)
{
    uint32_t r[4];
    draw(seed, index, frame, filter, purpose, 0, r);
    uint64_t r64 = ((uint64_t)r[1] << 32) | (uint64_t)r[0];
    return (uint64_t)(((u128)r64 * (u128)Q) >> 64);
}

/* anc_out[j] = base + parent of ticket j, for n tickets over the n_in weights q */
int orc_systematic(int64_t n_in, const uint64_t *q, int64_t n_tickets, uint64_t u,
                   int64_t base, int32_t *anc_out, int64_t *offspring)
{
    uint64_t C = 0, Q = 0;
    for (int64_t i = 0; i < n_in; ++i)
        Q += q[i];
    if (Q == 0)
        return ORC_EDEGENERATE;
    int64_t prev = 0;
    for (int64_t i = 0; i < n_in; ++i) {
        C += q[i];
        int64_t T = orc_tickets_below(C, n_tickets, u, Q);
        if (offspring)
            offspring[i] = T - prev;
        for (int64_t j = prev; j < T; ++j)
            anc_out[j] = (int32_t)(base + i);
        prev = T;
    }
    return prev == n_tickets ? ORC_OK : ORC_EINTERNAL;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4 schedulers.  count[g] = offspring of group g, target[g] = balanced */
/* size.  Senders: count > target (surplus), receivers: count < target.      */
/* GS (Alg. 2): senders and receivers in group order; each sender fills the  */
/* current receiver, moving on when the receiver is full, until the sender    */
/* is empty.  SGS (Alg. 3): both lists sorted by amount, descending (ties by  */
/* group index), then GS.  LGS (Alg. 4): sorted as SGS, the i-th sender is    */
/* paired with the i-th receiver for i < min(|S|,|R|), moving                 */
/* min(surplus, deficit).                                                     */
/* Returns the number of links written to (src, dst, cnt) in schedule order. */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t amount; int32_t group; } orc_entry;

static int entry_desc(const void *a, const void *b)
{
    const orc_entry *x = (const orc_entry *)a, *y = (const orc_entry *)b;
    if (x->amount != y->amount)
        return x->amount > y->amount ? -1 : 1;
    return x->group < y->group ? -1 : (x->group > y->group);
}

int64_t orc_schedule(int scheme, int32_t G, const int64_t *count, const int64_t *target,
                     int32_t *src, int32_t *dst, int64_t *cnt)
{
    orc_entry *S = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(G > 0 ? G : 1));
    orc_entry *R = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(G > 0 ? G : 1));
    int32_t nS = 0, nR = 0;
    for (int32_t g = 0; g < G; ++g) {
        if (count[g] > target[g]) { S[nS].amount = count[g] - target[g]; S[nS].group = g; ++nS; }
        if (count[g] < target[g]) { R[nR].amount = target[g] - count[g]; R[nR].group = g; ++nR; }
    }
    if (scheme != ORC_RPA_GS) {
        qsort(S, (size_t)nS, sizeof(orc_entry), entry_desc);
        qsort(R, (size_t)nR, sizeof(orc_entry), entry_desc);
    }
    int64_t L = 0;
    if (scheme == ORC_RPA_LGS) {
        int32_t C = nS < nR ? nS : nR;
        for (int32_t i = 0; i < C; ++i) {
            int64_t a = S[i].amount < R[i].amount ? S[i].amount : R[i].amount;
            src[L] = S[i].group; dst[L] = R[i].group; cnt[L] = a; ++L;
        }
    } else {
        int32_t j = 0;
        for (int32_t i = 0; i < nS; ++i) {
            int64_t left = S[i].amount;
            while (left > 0 && j < nR) {
                int64_t take = left < R[j].amount ? left : R[j].amount;
                src[L] = S[i].group; dst[L] = R[j].group; cnt[L] = take; ++L;
                left -= take;
                R[j].amount -= take;
                if (R[j].amount == 0)
                    ++j;
            }
        }
    }
    free(S);
    free(R);
    return L;
}

/* balanced partition of N into G groups: the first N mod G get one more */
void orc_balanced_offsets(int64_t N, int32_t G, int64_t *off)
{
    int64_t base = N / G, extra = N % G;
    off[0] = 0;
    for (int32_t g = 0; g < G; ++g)
        off[g + 1] = off[g] + base + (g < extra ? 1 : 0);
}

/* ------------------------------------------------------------------------ */
/* Resampling of all N particles held in the current group layout           */
/* goff_in[0..G].  Writes the ancestor of every new slot, the new layout     */
/* goff_out and each new slot's post-resampling log-weight lw_reset.         */
/*   ORC_SYSTEMATIC      global systematic (Alg. 1), weights reset (lw = 0). */
/*   ORC_RPA_GS/SGS/LGS  the same global tickets (proportional allocation,   */
/*                       one global offset, so the ancestors do not depend on */
/*                       G); group g keeps its first offspring, its surplus   */
/*                       (the last ones) is routed to receivers per schedule. */
/*   ORC_RPA2_GS/SGS/LGS two-stage proportional allocation (Bolic et al.):    */
/*                       stage 1 gives group g the N_g global tickets of its  */
/*                       cumulative range, as RPA does; stage 2 draws those   */
/*                       N_g offspring inside the group by its own systematic */
/*                       draw (offset from Philox(seed; g, k, filter, GROUP)) */
/*                       over the group's fixed-point weights; routing as RPA.*/
/*   ORC_RNA             each group resamples its own slots from its own      */
/*                       weights with its own offset; the offspring carry the */
/*                       group weight log(W_g / n_g); then the last           */
/*                       floor(alpha * min_g n_g) slots of group g move to     */
/*                       group g+1 (ring).                                    */
/* lw: float32 log-weights (the value the quantiser sees).                   */
/* lw_sum: per-particle log-weights used for the RNA group weights (FP64).   */
/* stats: links, moved, max group size, min group size.                      */
/* ------------------------------------------------------------------------ */
/* RNA local resampling and ring exchange (Sec. 3): every group resamples its
 * own slots from its own fixed-point weights with its own offset, the
 * offspring carry the group weight log(W_g / n_g) (FP64), and the last mig
 * offspring of group g go to the last mig slots of group succ[g]. */
static int rna_exchange(const orc_model *m, int64_t N, int32_t frame, int32_t G, const int64_t *goff_in,
                        const float *lw, const double *lw_sum, int64_t mig, const int32_t *succ,
                        int32_t *anc, double *lw_reset)
{
    int rc = ORC_OK;
    int64_t maxsz = 0;
    for (int32_t g = 0; g < G; ++g)
        if (goff_in[g + 1] - goff_in[g] > maxsz)
            maxsz = goff_in[g + 1] - goff_in[g];
    /* group log-weights log W_g = log sum_g e^lw - log sum e^lw, in FP64 */
    double Mall = -INFINITY;
    for (int64_t i = 0; i < N; ++i)
        if (lw_sum[i] > Mall) Mall = lw_sum[i];
    double tot = 0.0;
    for (int64_t i = 0; i < N; ++i)
        tot += exp(lw_sum[i] - Mall);
    const double log_tot = Mall + log(tot);
    int32_t *local = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxsz > 0 ? maxsz : 1));
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(maxsz > 0 ? maxsz : 1));
    for (int32_t g = 0; g < G; ++g) {
        int64_t lo = goff_in[g], sz = goff_in[g + 1] - lo;
        if (sz == 0)
            continue;
        float Mg = -INFINITY;
        double Mgd = -INFINITY;
        for (int64_t i = 0; i < sz; ++i) {
            if (lw[lo + i] > Mg) Mg = lw[lo + i];
            if (lw_sum[lo + i] > Mgd) Mgd = lw_sum[lo + i];
        }
        int s = orc_scale_bits(sz);
        uint64_t Q = 0;
        for (int64_t i = 0; i < sz; ++i) {
            q[i] = orc_quantise(lw[lo + i], Mg, s);
            Q += q[i];
        }
        double lwg;
        if (Q == 0) {
            /* every weight of the group is zero: it keeps its slots */
            for (int64_t i = 0; i < sz; ++i)
                local[i] = (int32_t)(lo + i);
            lwg = -INFINITY;
        } else {
            uint64_t u = orc_ticket_offset(m->seed, m->filter_id, (uint32_t)frame,
                                           ORC_PURPOSE_GROUP_RESAMPLE, (uint32_t)g, Q);
            int r2 = orc_systematic(sz, q, sz, u, lo, local, NULL);
            if (r2 != ORC_OK) { rc = r2; break; }
            double sg = 0.0;
            for (int64_t i = 0; i < sz; ++i)
                sg += exp(lw_sum[lo + i] - Mgd);
            lwg = (Mgd + log(sg)) - log_tot - log((double)sz);
        }
        int32_t gn = succ[g];
        int64_t gn_lo = goff_in[gn], gn_sz = goff_in[gn + 1] - gn_lo;
        for (int64_t s2 = 0; s2 < sz; ++s2) {
            int64_t slot;
            if (s2 < sz - mig)
                slot = lo + s2;
            else
                slot = gn_lo + gn_sz - mig + (s2 - (sz - mig));
            anc[slot] = local[s2];
            lw_reset[slot] = lwg;
        }
    }
    free(local);
    free(q);
    return rc;
}

static void group_extents(int32_t G, const int64_t *goff, int64_t *mx, int64_t *mn)
{
    *mx = 0;
    *mn = INT64_MAX;
    for (int32_t g = 0; g < G; ++g) {
        int64_t sz = goff[g + 1] - goff[g];
        if (sz > *mx) *mx = sz;
        if (sz < *mn) *mn = sz;
    }
}

int orc_resample(const orc_model *m, int scheme, double alpha, int64_t N, int32_t frame,
                 int32_t G, const int64_t *goff_in, const float *lw, const double *lw_sum,
                 int32_t *anc, double *lw_reset, int64_t *goff_out, int64_t stats[4])
{
    int rc = ORC_OK;
    stats[0] = stats[1] = 0;
    if (scheme == ORC_RNA) {
        int64_t minsz, maxsz;
        group_extents(G, goff_in, &maxsz, &minsz);
        int64_t mig = (int64_t)floor(alpha * (double)minsz);
        int32_t *succ = (int32_t *)calloc((size_t)(G > 0 ? G : 1), sizeof(int32_t));
        for (int32_t g = 0; g < G; ++g)
            succ[g] = (g + 1) % G;
        rc = rna_exchange(m, N, frame, G, goff_in, lw, lw_sum, mig, succ, anc, lw_reset);
        free(succ);
        for (int32_t g = 0; g <= G; ++g)
            goff_out[g] = goff_in[g];
        stats[0] = (G > 1 && mig > 0) ? G : 0; /* ring links that carry particles */
        stats[1] = G > 1 ? mig * G : 0;
        stats[2] = maxsz;
        stats[3] = minsz;
        return rc;
    }

    /* global systematic tickets */
    float M = -INFINITY;
    for (int64_t i = 0; i < N; ++i)
        if (lw[i] > M) M = lw[i];
    int s = orc_scale_bits(N);
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t Q = 0;
    for (int64_t i = 0; i < N; ++i) {
        q[i] = orc_quantise(lw[i], M, s);
        Q += q[i];
    }
    if (Q == 0) {
        /* no usable weight at all: keep every particle and its weight */
        for (int64_t i = 0; i < N; ++i) {
            anc[i] = (int32_t)i;
            lw_reset[i] = lw_sum[i];
        }
        for (int32_t g = 0; g <= G; ++g)
            goff_out[g] = goff_in[g];
        free(q);
        return ORC_EDEGENERATE;
    }
    uint64_t u = orc_ticket_offset(m->seed, m->filter_id, (uint32_t)frame, ORC_PURPOSE_RESAMPLE, 0u, Q);
    int32_t *sys = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    rc = orc_systematic(N, q, N, u, 0, sys, NULL);
    if (rc != ORC_OK || scheme == ORC_SYSTEMATIC) {
        if (rc == ORC_OK) {
            memcpy(anc, sys, sizeof(int32_t) * (size_t)N);
            for (int64_t i = 0; i < N; ++i)
                lw_reset[i] = 0.0;
            for (int32_t g = 0; g <= G; ++g)
                goff_out[g] = goff_in[g];
            int64_t mx = 0, mn = INT64_MAX;
            for (int32_t g = 0; g < G; ++g) {
                int64_t sz = goff_in[g + 1] - goff_in[g];
                if (sz > mx) mx = sz;
                if (sz < mn) mn = sz;
            }
            stats[2] = mx;
            stats[3] = mn;
        }
        free(q);
        free(sys);
        return rc;
    }

    /* RPA: offspring per group = tickets inside the group's cumulative range */
    const int two_stage = (scheme >= ORC_RPA2_GS && scheme <= ORC_RPA2_LGS);
    const int sched = two_stage ? scheme - (ORC_RPA2_GS - ORC_RPA_GS) : scheme;
    int64_t *T = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G + 1));
    int64_t *cnt_g = (int64_t *)malloc(sizeof(int64_t) * (size_t)G);
    int64_t *tgt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G + 1));
    uint64_t C = 0;
    T[0] = 0;
    for (int32_t g = 0; g < G; ++g) {
        for (int64_t i = goff_in[g]; i < goff_in[g + 1]; ++i)
            C += q[i];
        T[g + 1] = orc_tickets_below(C, N, u, Q);
        cnt_g[g] = T[g + 1] - T[g];
    }
    if (two_stage) {
        /* stage 2: group g's tickets T[g] .. T[g+1]-1 come from its own draw */
        for (int32_t g = 0; g < G && rc == ORC_OK; ++g) {
            if (cnt_g[g] == 0)
                continue;
            const int64_t lo = goff_in[g], sz = goff_in[g + 1] - lo;
            uint64_t Qg = 0;
            for (int64_t i = 0; i < sz; ++i)
                Qg += q[lo + i];
            const uint64_t ug = orc_ticket_offset(m->seed, m->filter_id, (uint32_t)frame,
                                                  ORC_PURPOSE_GROUP_RESAMPLE, (uint32_t)g, Qg);
            rc = orc_systematic(sz, q + lo, cnt_g[g], ug, lo, sys + T[g], NULL);
        }
    }
    orc_balanced_offsets(N, G, tgt);
    int64_t *target = (int64_t *)malloc(sizeof(int64_t) * (size_t)G);
    for (int32_t g = 0; g < G; ++g)
        target[g] = tgt[g + 1] - tgt[g];
    int32_t *lsrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * G + 1));
    int32_t *ldst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * G + 1));
    int64_t *lcnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * G + 1));
    int64_t L = orc_schedule(sched, G, cnt_g, target, lsrc, ldst, lcnt);
    int64_t *sent = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    int64_t *recv = (int64_t *)calloc((size_t)G, sizeof(int64_t));
    int64_t moved = 0;
    for (int64_t l = 0; l < L; ++l) {
        sent[lsrc[l]] += lcnt[l];
        recv[ldst[l]] += lcnt[l];
        moved += lcnt[l];
    }
    /* new layout */
    goff_out[0] = 0;
    for (int32_t g = 0; g < G; ++g)
        goff_out[g + 1] = goff_out[g] + cnt_g[g] - sent[g] + recv[g];
    /* kept offspring: the first cnt_g - sent tickets of the group */
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)G);
    int64_t *sendpos = (int64_t *)malloc(sizeof(int64_t) * (size_t)G);
    for (int32_t g = 0; g < G; ++g) {
        int64_t keep = cnt_g[g] - sent[g];
        for (int64_t t = 0; t < keep; ++t)
            anc[goff_out[g] + t] = sys[T[g] + t];
        fill[g] = keep;
        sendpos[g] = T[g] + keep; /* the surplus tickets follow the kept ones */
    }
    /* routed offspring, in schedule order */
    for (int64_t l = 0; l < L; ++l) {
        int32_t a = lsrc[l], b = ldst[l];
        for (int64_t t = 0; t < lcnt[l]; ++t)
            anc[goff_out[b] + fill[b] + t] = sys[sendpos[a] + t];
        fill[b] += lcnt[l];
        sendpos[a] += lcnt[l];
    }
    for (int64_t i = 0; i < N; ++i)
        lw_reset[i] = 0.0;
    int64_t mx = 0, mn = INT64_MAX;
    for (int32_t g = 0; g < G; ++g) {
        int64_t sz = goff_out[g + 1] - goff_out[g];
        if (sz > mx) mx = sz;
        if (sz < mn) mn = sz;
    }
    stats[0] = L;
    stats[1] = moved;
    stats[2] = mx;
    stats[3] = mn;
    free(T); free(cnt_g); free(tgt); free(target); free(lsrc); free(ldst); free(lcnt);
    free(sent); free(recv); free(fill); free(sendpos); free(q); free(sys);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* ARNA (Sec. 7): RNA whose exchange ratio follows the number of groups      */
/* involved in tracking and whose ring order is redrawn when the object is   */
/* lost.  The paper describes ARNA in words only; this is the reading taken: */
/*   involved   group g is involved when proportional allocation (the global */
/*              systematic tickets of RPA over its cumulative range) gives   */
/*              it at least its own size: o_g >= n_g (exact integers; none   */
/*              when no weight is usable).                                   */
/*   ratio      alpha_k = alpha (1 - |I| / G), alpha the caller's maximum;    */
/*              mig = floor(alpha (G - |I|) min_g n_g / G), evaluated in     */
/*              FP64 in that order.                                          */
/*   ring       a permutation of the groups kept between frames; group       */
/*              ring[p] sends its last mig offspring to ring[(p+1) mod G].    */
/*   lost       decided by the caller (the frame's log-evidence below zero:  */
/*              the cloud explains the frame no better than the background). */
/*              Then the ring is redrawn before the exchange: the groups in  */
/*              increasing order of the first Philox word of (seed; g,      */
/*              frame, filter, RING), ties by group index.                   */
/* stats: links, moved, max group size, min group size, involved groups.    */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t key; int32_t group; } orc_ring_key;

static int ring_key_asc(const void *a, const void *b)
{
    const orc_ring_key *x = (const orc_ring_key *)a, *y = (const orc_ring_key *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return x->group < y->group ? -1 : (x->group > y->group);
}

void orc_arna_ring(uint64_t seed, uint32_t filter, uint32_t frame, int32_t G, int32_t *ring)
{
    orc_ring_key *k = (orc_ring_key *)malloc(sizeof(orc_ring_key) * (size_t)(G > 0 ? G : 1));
    for (int32_t g = 0; g < G; ++g) {
        uint32_t r[4];
        draw(seed, (uint32_t)g, frame, filter, ORC_PURPOSE_RING, 0, r);
        k[g].key = r[0];
        k[g].group = g;
    }
    qsort(k, (size_t)G, sizeof(orc_ring_key), ring_key_asc);
    for (int32_t p = 0; p < G; ++p)
        ring[p] = k[p].group;
    free(k);
}

int orc_resample_arna(const orc_model *m, double alpha, int64_t N, int32_t frame, int32_t G,
                      const int64_t *goff_in, const float *lw, const double *lw_sum, int32_t lost,
                      int32_t *ring, int32_t *anc, double *lw_reset, int64_t *goff_out, int64_t stats[5])
{
    /* offspring of every group under proportional allocation */
    float M = -INFINITY;
    for (int64_t i = 0; i < N; ++i)
        if (lw[i] > M) M = lw[i];
    const int s = orc_scale_bits(N);
    uint64_t Q = 0;
    for (int64_t i = 0; i < N; ++i)
        Q += orc_quantise(lw[i], M, s);
    int32_t involved = 0;
    if (Q > 0) {
        const uint64_t u = orc_ticket_offset(m->seed, m->filter_id, (uint32_t)frame, ORC_PURPOSE_RESAMPLE, 0u, Q);
        uint64_t C = 0;
        int64_t below = 0;
        for (int32_t g = 0; g < G; ++g) {
            for (int64_t i = goff_in[g]; i < goff_in[g + 1]; ++i)
                C += orc_quantise(lw[i], M, s);
            const int64_t t = orc_tickets_below(C, N, u, Q);
            if (t - below >= goff_in[g + 1] - goff_in[g])
                ++involved;
            below = t;
        }
    }
    int64_t minsz, maxsz;
    group_extents(G, goff_in, &maxsz, &minsz);
    const int64_t mig = (int64_t)floor(alpha * (double)(G - involved) * (double)minsz / (double)G);
    if (lost)
        orc_arna_ring(m->seed, m->filter_id, (uint32_t)frame, G, ring);
    int32_t *succ = (int32_t *)calloc((size_t)(G > 0 ? G : 1), sizeof(int32_t));
    for (int32_t p = 0; p < G; ++p)
        succ[ring[p]] = ring[(p + 1) % G];
    const int rc = rna_exchange(m, N, frame, G, goff_in, lw, lw_sum, mig, succ, anc, lw_reset);
    free(succ);
    for (int32_t g = 0; g <= G; ++g)
        goff_out[g] = goff_in[g];
    stats[0] = (G > 1 && mig > 0) ? G : 0;
    stats[1] = G > 1 ? mig * G : 0;
    stats[2] = maxsz;
    stats[3] = minsz;
    stats[4] = involved;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* A whole SIR run (Alg. 1): init, then for each frame propagate, weight,    */
/* summarise, resample (when N_eff < ess_threshold; +inf: every frame).     */
/* frames: K x H x W doubles.  est: K x 8 (mean[5],                          */
/* log-evidence, ess, max lw).  st (6N) holds the last weighted particles.   */
/* ------------------------------------------------------------------------ */
int orc_run(const orc_model *m, int64_t N, int32_t group_size, int scheme, double alpha,
            double ess_threshold, int32_t K, const double *frames, double *est, double *st_out)
{
    int32_t G = (int32_t)((N + group_size - 1) / group_size);
    double *cur = (double *)malloc(sizeof(double) * (size_t)(6 * N));
    double *nxt = (double *)malloc(sizeof(double) * (size_t)(6 * N));
    double *lw_prev = (double *)malloc(sizeof(double) * (size_t)N);
    float *lwf = (float *)malloc(sizeof(float) * (size_t)N);
    int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t *goff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G + 1));
    int64_t *goff2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G + 1));
    int32_t *ring = (int32_t *)malloc(sizeof(int32_t) * (size_t)G);  /* ARNA ring order, identity at start */
    for (int32_t g = 0; g < G; ++g)
        ring[g] = g;
    int rc = ORC_OK;
    orc_init(m, N, cur);
    orc_balanced_offsets(N, G, goff);
    for (int64_t i = 0; i < N; ++i) {
        anc[i] = (int32_t)i;
        lw_prev[i] = cur[5 * N + i];
    }
    const int64_t npix = (int64_t)m->width * m->height;
    for (int32_t k = 0; k < K; ++k) {
        orc_propagate(m, N, k + 1, cur, anc, lw_prev, nxt);
        orc_weight(m, N, frames + (int64_t)k * npix, nxt);
        orc_summary(N, nxt, lw_prev, est + 8 * (int64_t)k);
        /* Alg. 1: resample only while the effective sample size is below
         * the threshold; otherwise keep the particles and carry the weights */
        if (!(est[8 * (int64_t)k + 6] < ess_threshold)) {
            for (int64_t i = 0; i < N; ++i) {
                anc[i] = (int32_t)i;
                lw_prev[i] = nxt[5 * N + i];
            }
        } else {
            for (int64_t i = 0; i < N; ++i)
                lwf[i] = (float)nxt[5 * N + i];
            int64_t stats[5];
            if (scheme == ORC_ARNA) {
                const int32_t lost = !(est[8 * (int64_t)k + 5] >= 0.0);
                rc = orc_resample_arna(m, alpha, N, k + 1, G, goff, lwf, nxt + 5 * N, lost, ring, anc, lw_prev,
                                       goff2, stats);
            } else {
                rc = orc_resample(m, scheme, alpha, N, k + 1, G, goff, lwf, nxt + 5 * N, anc, lw_prev, goff2,
                                  stats);
            }
            if (rc != ORC_OK)
                break;
            memcpy(goff, goff2, sizeof(int64_t) * (size_t)(G + 1));
        }
        double *t = cur; cur = nxt; nxt = t;
    }
    if (st_out)
        memcpy(st_out, cur, sizeof(double) * (size_t)(6 * N));
    free(cur); free(nxt); free(lw_prev); free(lwf); free(anc); free(goff); free(goff2); free(ring);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the log marginal likelihood estimate (the sum of the per-    */
/* frame log-evidences of Alg. 1 with systematic resampling every frame)    */
/* with respect to theta = (sigma_PSF, A, I_bg, sigma_m), the intensity     */
/* fixed at I0 = A.  Resampling is a stop-gradient: the ancestors are held  */
/* fixed; the patch anchors too (the objective is piecewise smooth in the   */
/* positions).  Reverse mode, FP64.                                         */
/* ------------------------------------------------------------------------ */

/* l and its partials for one particle, from eq. 3/eq. 4 pixel by pixel:
 * out = {l, dl/dsigma, dl/dI0, dl/dbg, dl/dx, dl/dy}.  (ax, ay) forces the
 * anchor when ax != INT32_MIN. */
void orc_loglik_partials(const orc_model *m, const double *frame, double x, double y, double I0, int32_t ax,
                         int32_t ay, double out[6])
{
    for (int c = 0; c < 6; ++c)
        out[c] = 0.0;
    if (!isfinite(x) || !isfinite(y) || !isfinite(I0)) {
        out[0] = -INFINITY;
        return;
    }
    const int r = m->patch_radius;
    int64_t cx, cy;
    if (ax != INT32_MIN) {
        cx = ax;
        cy = ay;
    } else {
        const double cxd = floor(x + 0.5), cyd = floor(y + 0.5);
        if (cxd < -r - 1.0 || cxd > m->width + r || cyd < -r - 1.0 || cyd > m->height + r)
            return;
        cx = (int64_t)cxd;
        cy = (int64_t)cyd;
    }
    const double s = m->psf_sigma, s2 = s * s, sx2 = m->sigma_xi * m->sigma_xi;
    for (int64_t py = cy - r; py <= cy + r; ++py) {
        if (py < 0 || py >= m->height)
            continue;
        for (int64_t px = cx - r; px <= cx + r; ++px) {
            if (px < 0 || px >= m->width)
                continue;
            const double dx = (double)px - x, dy = (double)py - y, d2 = dx * dx + dy * dy;
            const double g = exp(-d2 / (2.0 * s2));
            const double I = I0 * g + m->background;
            const double z = frame[py * (int64_t)m->width + px];
            const double res = z - I, res0 = z - m->background;
            out[0] += -(res * res - res0 * res0) / (2.0 * sx2);
            const double dl_dI = res / sx2;               /* d l / d I at this pixel */
            out[1] += dl_dI * I0 * g * d2 / (s2 * s);     /* dI/dsigma = I0 g d^2 / s^3 */
            out[2] += dl_dI * g;                          /* dI/dI0 = g */
            out[3] += (res - res0) / sx2;                 /* I and res0 both move with I_bg */
            out[4] += dl_dI * I0 * g * dx / s2;           /* dI/dx = I0 g (px - x) / s^2 */
            out[5] += dl_dI * I0 * g * dy / s2;
        }
    }
}

/* K frames from the prior: L = sum_k [log sum_i e^{l_k^i} - log N] and dL/dtheta.
 * theta overrides (psf_sigma, amplitude, background, sigma_m) of m.
 * anc_io (K x N): if replay, slot i of frame k+1 (k = 0..K-1) takes anc_io[k N + i]
 * (row 0 is the identity of the first step); otherwise it is written.  anchor_io
 * (K x 2 x N: cx then cy per frame): replayed or written likewise. */
int orc_grad_run(const orc_model *m0, int64_t N, int32_t K, const double *frames, const double theta[4],
                 int replay, int32_t *anc_io, int32_t *anchor_io, double *L_out, double grad[4])
{
    orc_model m = *m0;
    m.psf_sigma = theta[0];
    m.amplitude = theta[1];
    m.background = theta[2];
    m.sigma_m = theta[3];
    const double A = theta[1];
    const int64_t npix = (int64_t)m.width * m.height;
    double *cur = (double *)malloc(sizeof(double) * (size_t)(6 * N));
    double *nxt = (double *)malloc(sizeof(double) * (size_t)(6 * N));
    double *zero = (double *)calloc((size_t)N, sizeof(double));
    double *wlx = (double *)malloc(sizeof(double) * (size_t)(K * N)); /* w dl/dx per frame */
    double *wly = (double *)malloc(sizeof(double) * (size_t)(K * N));
    double *lam = (double *)calloc((size_t)N, sizeof(double));
    double *mu = (double *)calloc((size_t)N, sizeof(double));
    double *lam2 = (double *)malloc(sizeof(double) * (size_t)N);
    double *mu2 = (double *)malloc(sizeof(double) * (size_t)N);
    double *part = (double *)malloc(sizeof(double) * (size_t)(6 * N));
    int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int rc = ORC_OK;
    double L = 0.0, gd[3] = {0, 0, 0};
    orc_init(&m, N, cur);
    for (int64_t i = 0; i < N; ++i)
        anc[i] = (int32_t)i;
    int32_t G = 1;
    int64_t goff[2] = {0, N}, goff2[2];
    for (int32_t k = 0; k < K && rc == ORC_OK; ++k) {
        if (replay)
            memcpy(anc, anc_io + (int64_t)k * N, sizeof(int32_t) * (size_t)N);
        else
            memcpy(anc_io + (int64_t)k * N, anc, sizeof(int32_t) * (size_t)N);
        orc_propagate(&m, N, k + 1, cur, anc, zero, nxt);
        const double *fr = frames + (int64_t)k * npix;
        int32_t *an = anchor_io + (int64_t)k * 2 * N;
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t i = 0; i < N; ++i) {
            int32_t ax = INT32_MIN, ay = INT32_MIN;
            if (replay) {
                ax = an[i];
                ay = an[N + i];
            }
            orc_loglik_partials(&m, fr, nxt[i], nxt[N + i], A, ax, ay, part + 6 * i);
            if (!replay) {
                an[i] = (int32_t)floor(nxt[i] + 0.5);
                an[N + i] = (int32_t)floor(nxt[N + i] + 0.5);
            }
            nxt[5 * N + i] = part[6 * i];
        }
        double M = -INFINITY;
        for (int64_t i = 0; i < N; ++i)
            if (part[6 * i] > M)
                M = part[6 * i];
        /* the exponentials in parallel, the sums serially in particle order */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i)
            lam2[i] = exp(nxt[5 * N + i] - M);
        double tot = 0.0;
        for (int64_t i = 0; i < N; ++i)
            tot += lam2[i];
        L += M + log(tot) - log((double)N);
        for (int64_t i = 0; i < N; ++i) {
            const double w = lam2[i] / tot;
            gd[0] += w * part[6 * i + 1];
            gd[1] += w * part[6 * i + 2];
            gd[2] += w * part[6 * i + 3];
            wlx[(int64_t)k * N + i] = w * part[6 * i + 4];
            wly[(int64_t)k * N + i] = w * part[6 * i + 5];
        }
        if (k + 1 < K && !replay) {
            float *lwf = (float *)malloc(sizeof(float) * (size_t)N);
            double *lwr = (double *)malloc(sizeof(double) * (size_t)N);
            int64_t st[4];
            for (int64_t i = 0; i < N; ++i)
                lwf[i] = (float)nxt[5 * N + i];
            rc = orc_resample(&m, ORC_SYSTEMATIC, 0.0, N, k + 1, G, goff, lwf, nxt + 5 * N, anc, lwr, goff2, st);
            free(lwf);
            free(lwr);
        }
        double *t = cur;
        cur = nxt;
        nxt = t;
    }
    /* reverse sweep over the position adjoints: x_{k+1}^c = x_k^{a(c)} + ... so
     * the adjoint of x_k^i collects w_k^i dl/dx plus the adjoints of its children */
    double gsm = 0.0;
    for (int32_t k = K - 1; k >= 0 && rc == ORC_OK; --k) {
        for (int64_t i = 0; i < N; ++i) {
            lam2[i] = wlx[(int64_t)k * N + i];
            mu2[i] = wly[(int64_t)k * N + i];
        }
        if (k + 1 < K) {
            const int32_t *a = anc_io + (int64_t)(k + 1) * N;
            for (int64_t c = 0; c < N; ++c) {
                lam2[a[c]] += lam[c];
                mu2[a[c]] += mu[c];
            }
        }
        /* the normals in parallel, the sum serially in particle order */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double e[5];
            orc_normals5(m.seed, (uint32_t)i, (uint32_t)(k + 1), m.filter_id, e);
            part[2 * i] = e[0];
            part[2 * i + 1] = e[1];
        }
        for (int64_t i = 0; i < N; ++i)
            gsm += lam2[i] * part[2 * i] + mu2[i] * part[2 * i + 1];  /* dx/dsigma_m = e1, dy/dsigma_m = e2 */
        double *t = lam; lam = lam2; lam2 = t;
        t = mu; mu = mu2; mu2 = t;
    }
    *L_out = L;
    grad[0] = gd[0];
    grad[1] = gd[1];
    grad[2] = gd[2];
    grad[3] = gsm;
    free(cur); free(nxt); free(zero); free(wlx); free(wly); free(lam); free(mu); free(lam2); free(mu2);
    free(part); free(anc);
    return rc;
}
