// ppf_resample.cu -- the resampling step of Alg. 1 on 64-bit fixed-point
// weights, and the distributed schemes of Sec. 3-4 mapped onto particle groups:
//   systematic  one global offset u, ticket j at (u + jQ)/N of the cumulative
//               weight; the parent of ticket j is the first particle whose
//               cumulative weight C_i satisfies N C_i > u + jQ.
//   RPA         the same global tickets (proportional allocation); group g
//               holds the tickets of its own cumulative range, keeps the first
//               ones and routes its surplus to receivers following the Greedy
//               (Alg. 2), Sorted Greedy (Alg. 3) or Largest Gradient (Alg. 4)
//               schedule.
//   RNA         every group resamples its own slots from its own weights with
//               its own offset (non-proportional allocation); its offspring
//               carry the group weight, and the last floor(alpha min n_g) slots
//               of every group migrate to the next group of the ring.
// Every resampling kernel takes the N_eff threshold of Alg. 1: when the
// step's effective sample size is not below it, the kernels do nothing but
// mark the particles as kept (the next step carries their weights).
#include <cmath>

#include "ppf_device.cuh"
#include "ppf_internal.h"
#include "ppf_tiles.cuh"

namespace ppf {

// Alg. 1 resamples only while N_eff < N_threshold (NaN N_eff: resample, which
// then reports the degenerate weights).
__device__ __forceinline__ bool kept_by_ess(const DevSummary *sum, double ess_thr)
{
    return sum->ess >= ess_thr;
}

// Balanced layout: group g holds n_g = q + [g < r] slots, q = floor(N/G) and
// r = N mod G (divided once on the host: 64-bit division is a long software
// sequence on the device), starting at off_g = g q + min(g, r).
struct Balanced {
    int64_t q, r;
};

inline Balanced balanced_layout(int64_t N, int32_t G)
{
    return Balanced{N / G, N % G};
}

__device__ __forceinline__ int64_t target_of(const Balanced &b, int32_t g)
{
    return b.q + ((int64_t)g < b.r ? 1 : 0);
}

__device__ __forceinline__ int64_t balanced_offset(const Balanced &b, int32_t g)
{
    return (int64_t)g * b.q + ((int64_t)g < b.r ? (int64_t)g : b.r);
}

// ---------------------------------------------------------------- R1 tiles
// Tile totals Q_t: every thread loads its four float4 (coalesced, all in
// flight together), then quantises them two at a time; one block sum.  No
// shared buffer, so more blocks fit an SM.
__global__ void __launch_bounds__(TILE_THREADS, 5) tile_totals_kernel(const float *__restrict__ lw, int64_t N,
                                                                      const DevSummary *__restrict__ sum,
                                                                      double ess_thr, uint64_t *__restrict__ Qt)
{
    // Blocks take tiles blockIdx.x, + gridDim.x, ... (one each when the grid
    // has a block per tile).  A full, aligned tile's loads go out one tile
    // ahead, so that they are in flight while the block quantises the tile
    // before and waits at its reduction.
    if (kept_by_ess(sum, ess_thr))
        return;
    constexpr int V = TILE / 4 / TILE_THREADS;
    __shared__ uint64_t wsum[TILE_THREADS / 32];
    const int64_t T = (N + TILE - 1) / TILE;
    const float M = sum->M;
    const int s = scale_bits(N);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto full_tile = [&](int64_t t) {
        const int64_t lo = t * TILE;
        return N - lo >= TILE && ((reinterpret_cast<uintptr_t>(lw + lo) & 15) == 0);
    };
    auto load = [&](int64_t t, float4 (&v)[V]) {
        const float4 *v4 = reinterpret_cast<const float4 *>(lw + t * TILE) + threadIdx.x;
#pragma unroll
        for (int k = 0; k < V; ++k)
            v[k] = __ldg(v4 + k * TILE_THREADS);
    };
    int64_t t = blockIdx.x;
    float4 v[V];
    if (t < T && full_tile(t))
        load(t, v);
    for (; t < T; t += gridDim.x) {
        const int64_t tn = t + gridDim.x;
        float4 vn[V];
        if (tn < T && full_tile(tn))
            load(tn, vn);
        uint64_t acc = 0;
        if (full_tile(t)) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                uint64_t a, b, c, d;
                quantise2(v[k].x, v[k].y, M, s, a, b);
                quantise2(v[k].z, v[k].w, M, s, c, d);
                acc += a + b + c + d;
            }
        } else {
            const int64_t lo = t * TILE;
            const int n = (int)(N - lo < TILE ? N - lo : TILE);
            for (int e = threadIdx.x; e < n; e += blockDim.x)
                acc += quantise(__ldg(lw + lo + e), M, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0)
            wsum[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t total = 0;
            for (int w = 0; w < TILE_THREADS / 32; ++w)
                total += wsum[w];
            Qt[t] = total;
        }
        __syncthreads();  // wsum is rewritten for the next tile
#pragma unroll
        for (int k = 0; k < V; ++k)
            v[k] = vn[k];
    }
}

// Tile totals for RPA and ARNA, and for every group start inside the tile the
// local prefix before it.  A balanced layout puts one or two group starts in
// a tile: their prefixes are masked sums of the weights the threads already
// hold, reduced together with the total.  A tile with more starts (small
// groups, or the unequal groups LGS leaves) scans its weights in shared
// memory and reads the prefixes there.  Every tile also records the first
// group starting at or after it and how many start inside it (GT_MASKED + 1
// meaning more), for the fill's routing of kept tickets.
constexpr int GT_MASKED = 4;  // group starts per tile handled by masked sums

// The thread's part of the tile total (acc[GT_MASKED]) and of the prefix
// before each of the NS group starts at local positions spos[j] (acc[j]).
// Thread t holds the quads 4 (t + k TILE_THREADS) .. + 3: a quad lies wholly
// below or above a start except the one quad that holds it, so each start
// costs a select of the quad's sum, and the partial quad a few more.
template <int NS>
__device__ __forceinline__ void masked_sums(const float4 (&v)[TILE / 4 / TILE_THREADS], const int32_t *spos, float M,
                                            int s, uint64_t (&acc)[GT_MASKED + 1])
{
    constexpr int V = TILE / 4 / TILE_THREADS;
    int p[NS > 0 ? NS : 1];
#pragma unroll
    for (int j = 0; j < NS; ++j)
        p[j] = spos[j];
#pragma unroll
    for (int j = 0; j <= GT_MASKED; ++j)
        acc[j] = 0;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        uint64_t w0, w1, w2, w3;
        quantise2(v[k].x, v[k].y, M, s, w0, w1);
        quantise2(v[k].z, v[k].w, M, s, w2, w3);
        const uint64_t w01 = w0 + w1, qs = w01 + w2 + w3;
        acc[GT_MASKED] += qs;
        const int e0 = 4 * ((int)threadIdx.x + k * TILE_THREADS);
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const int d = p[j] - e0;  // elements of the quad below start j
            const uint64_t part = d >= 4 ? qs : (d == 3 ? w01 + w2 : (d == 2 ? w01 : (d == 1 ? w0 : 0ull)));
            acc[j] += d > 0 ? part : 0ull;
        }
    }
}

__global__ void __launch_bounds__(TILE_THREADS, 5) tile_group_totals_kernel(
    const float *__restrict__ lw, int64_t N, const DevSummary *__restrict__ sum, double ess_thr,
    uint64_t *__restrict__ Qt, const int64_t *__restrict__ goff, int32_t G, uint64_t *__restrict__ Cbl,
    int32_t *__restrict__ tile_g)
{
    if (kept_by_ess(sum, ess_thr))
        return;
    __shared__ uint64_t buf[TILE_SMEM_U64];
    __shared__ uint64_t red[33];
    __shared__ int32_t gfirst, nstart;
    __shared__ int32_t spos[GT_MASKED];
    __shared__ uint64_t wsum[TILE_THREADS / 32][GT_MASKED + 1];
    const int64_t lo = (int64_t)blockIdx.x * TILE;
    const int n = (int)(N - lo < TILE ? N - lo : TILE);
    // the weights first, so that their loads are in flight during the search
    // warp 0 does for the tile's group starts.  Thread t holds elements
    // 4 (t + k TILE_THREADS) + j, j < 4.
    constexpr int V = TILE / 4 / TILE_THREADS;
    const bool full = n == TILE && ((reinterpret_cast<uintptr_t>(lw + lo) & 15) == 0);
    float4 v[V];
    if (full) {
        const float4 *v4 = reinterpret_cast<const float4 *>(lw + lo) + threadIdx.x;
#pragma unroll
        for (int k = 0; k < V; ++k)
            v[k] = __ldg(v4 + k * TILE_THREADS);
    }
    if (threadIdx.x < 32) {
        // warp 0: the first g with goff[g] >= lo (goff[G] = N >= lo, so it
        // exists).  The first round probes the 32 groups around the balanced
        // layout's guess lo G / N, which holds the answer for a balanced
        // layout; otherwise 32-way rounds narrow [a, b] (invariant: the
        // answer lies in it) by a factor 32 each.
        const int lane = threadIdx.x;
        const int32_t guess = (int32_t)(lo * (int64_t)G / N);
        int32_t a = guess > 0 ? guess - 1 : 0, b = a + 31 < G ? a + 31 : G;
        {
            const int32_t p = a + lane;
            const unsigned m = __ballot_sync(0xffffffffu, p <= b && goff[p] >= lo);
            if (m & 1u) {          // goff[a] >= lo: the answer is at or before a
                b = a;
                a = 0;
            } else if (m != 0u) {  // the first lane at or past lo
                a = b = a + __ffs(m) - 1;
            } else {               // every probe below lo
                a = b + 1;
                b = G;
            }
        }
        while (a < b) {
            const int32_t step = (b - a + 30) / 31;  // 31 steps reach b
            const int32_t p = a + lane * step;
            const unsigned m = __ballot_sync(0xffffffffu, p <= b && goff[p] >= lo);
            if (m & 1u) {
                b = a;
            } else if (m != 0u) {
                const int f = __ffs(m) - 1;  // probes f - 1 below lo, f at or past it
                b = a + f * step;
                a = a + (f - 1) * step + 1;
            } else {
                const int last = (b - a) / step;  // the last probe (at or below b)
                a = a + last * step + 1;
            }
        }
        // the group starts inside the tile: lanes 0 .. GT_MASKED look at
        // goff[a + lane] (a prefix of them lie inside; lane GT_MASKED tells
        // whether there are more than GT_MASKED)
        const int32_t gg = a + lane;
        const bool inside = lane <= GT_MASKED && gg <= G && goff[gg] < lo + n;
        const unsigned mi = __ballot_sync(0xffffffffu, inside);
        const int ns = __popc(mi);
        if (inside && lane < GT_MASKED)
            spos[lane] = (int)(goff[gg] - lo);
        if (lane == 0) {
            gfirst = a;
            nstart = ns;
            tile_g[2 * blockIdx.x] = a;
            tile_g[2 * blockIdx.x + 1] = ns;
        }
    }
    __syncthreads();
    const int ns = nstart;
    const float M = sum->M;
    const int s = scale_bits(N);
    if (ns <= GT_MASKED && full) {
        uint64_t acc[GT_MASKED + 1];
        switch (ns) {  // uniform over the block: only the starts the tile has
        case 0: masked_sums<0>(v, spos, M, s, acc); break;
        case 1: masked_sums<1>(v, spos, M, s, acc); break;
        case 2: masked_sums<2>(v, spos, M, s, acc); break;
        case 3: masked_sums<3>(v, spos, M, s, acc); break;
        default: masked_sums<4>(v, spos, M, s, acc); break;
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int j = 0; j <= GT_MASKED; ++j) {
            if (j < ns || j == GT_MASKED) {
                uint64_t x = acc[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0)
                    wsum[warp][j] = x;
            }
        }
        __syncthreads();
        if (threadIdx.x <= GT_MASKED) {
            uint64_t x = 0;
            if (threadIdx.x < ns || threadIdx.x == GT_MASKED)
                for (int w = 0; w < TILE_THREADS / 32; ++w)
                    x += wsum[w][threadIdx.x];
            if (threadIdx.x == GT_MASKED)
                Qt[blockIdx.x] = x;
            else if (threadIdx.x < ns)
                Cbl[gfirst + threadIdx.x] = x;
        }
        return;
    }
    uint64_t q[TILE_ITEMS];
    tile_weights(lw, lo, n, M, s, buf, q);
    const uint64_t total = tile_scan(q, buf, red);
    if (threadIdx.x == 0)
        Qt[blockIdx.x] = total;
    __syncthreads();
    for (int32_t g = gfirst + threadIdx.x; g <= G; g += blockDim.x) {
        const int64_t pos = goff[g];
        if (pos >= lo + n)
            break;
        const int k = (int)(pos - lo);
        Cbl[g] = (k == 0) ? 0ull : buf[padc(k - 1)];
    }
}

// ---------------------------------------------------------------- R2 scan
// One block: exclusive tile prefix, total Q, ticket offset u, tickets below
// each tile start, fill work items (and the tile of each item when item_tile
// is given); for RPA (rpa = 1) and ARNA (rpa = 2) the tickets below each
// group start.  A proportional draw (rpa != 2) at a low N_eff also sets the
// next step to the direct likelihood path.  With prefix_only the kernel stops
// after the prefix and the draw (tile_tickets_kernel does the rest in
// parallel).
// When the T + 1 tile values fit the dynamic shared memory (T <= smem_tiles),
// they are loaded there with coalesced reads, and each of the two prefix sums
// gives every thread one contiguous segment: a local sum, one block scan,
// then the segment's prefixes.  Otherwise every array is walked in rounds of
// blockDim consecutive entries, each round closed by a block scan.
__global__ void __launch_bounds__(1024) tile_scan_kernel(
    int64_t N, int32_t T, const uint64_t *__restrict__ Qt, uint64_t *__restrict__ Ct, int64_t *__restrict__ Tt,
    int32_t *__restrict__ item_off, int32_t *__restrict__ item_tile, DevSummary *sum, double ess_thr, uint64_t seed,
    uint32_t fid, uint32_t frame, const int64_t *__restrict__ goff, int32_t G, int rpa,
    const uint64_t *__restrict__ Cbl, int64_t *__restrict__ Tg, int32_t smem_tiles, Divisor ndiv, int prefix_only,
    int2 *__restrict__ extra)
{
    extern __shared__ uint64_t sT[];  // (smem_tiles + 1) tile values
    __shared__ uint64_t red[33];
    __shared__ uint64_t su, s_qN;
    __shared__ uint32_t s_qR;
    if (threadIdx.x == 0) {
        sum->n_split = 0;  // the two-stage draw's split list is rebuilt after the scan
        sum->n_runs = 0;
        sum->n_extra = 0;  // and the fill's list of further ticket runs
    }
    if (kept_by_ess(sum, ess_thr)) {  // N_eff test: keep the particles and the layout
        if (threadIdx.x == 0) {
            sum->degenerate = 1;
            sum->flags |= FLAG_KEPT;
            sum->n_items = 0;
            sum->links = 0;
            sum->moved = 0;
        }
        return;
    }
    const bool in_smem = T <= smem_tiles;
    const int seg = (T + (int)blockDim.x - 1) / (int)blockDim.x;
    const int s0 = min(T, (int)threadIdx.x * seg), s1 = min(T, s0 + seg);
    uint64_t total = 0;
    if (in_smem) {
        for (int t = threadIdx.x; t < T; t += blockDim.x)
            sT[t] = __ldg(Qt + t);
        __syncthreads();
        uint64_t loc = 0;
        for (int t = s0; t < s1; ++t)
            loc += sT[t];
        uint64_t run = block_excl_scan_u64(loc, red, &total);
        for (int t = s0; t < s1; ++t) {
            const uint64_t v = sT[t];
            sT[t] = run;  // exclusive tile prefix
            run += v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < T; t += blockDim.x)
            Ct[t] = sT[t];
    } else {
        for (int base = 0; base < T; base += blockDim.x) {
            const int t = base + threadIdx.x;
            const uint64_t v = (t < T) ? Qt[t] : 0ull;
            uint64_t tot;
            const uint64_t ex = block_excl_scan_u64(v, red, &tot);
            if (t < T)
                Ct[t] = total + ex;
            total += tot;
        }
    }
    if (threadIdx.x == 0) {
        Ct[T] = total;
        const int deg = (total == 0ull);
        sum->degenerate = deg;
        if (deg)
            sum->flags |= FLAG_DEGENERATE;
        sum->Q = total;
        s_qN = total / (uint64_t)N;
        s_qR = (uint32_t)(total % (uint64_t)N);
        sum->qN = s_qN;
        sum->qR = s_qR;
        su = deg ? 0ull : ticket_offset(seed, fid, frame, PURPOSE_RESAMPLE, 0u, total);
        sum->u = su;
    }
    __syncthreads();
    const uint64_t Q = total, u = su;
    const TicketGrid tg = ticket_grid(Q, u, s_qN, s_qR, ndiv);
    if (Q == 0ull) {
        if (threadIdx.x == 0)
            sum->n_items = 0;
        return;
    }
    if (threadIdx.x == 0 && rpa != 2 && sum->ess < (double)N / BIN_CONCENTRATE)
        sum->bin_next = 0;  // a concentrating proportional draw: the next step is direct
    if (prefix_only) {  // tile_tickets_kernel takes it from here, one thread per tile and group
        if (threadIdx.x == 0) {
            sum->n_items = 0;
            if (!rpa) {
                sum->links = 0;
                sum->moved = 0;
            }
        }
        return;
    }
    for (int t = threadIdx.x; t <= T; t += blockDim.x) {
        const int64_t v = (t == T) ? N : tickets_below_grid(in_smem ? sT[t] : Ct[t], tg);
        Tt[t] = v;
        if (in_smem)
            sT[t] = (uint64_t)v;  // each thread rewrites only the entries it read
    }
    __syncthreads();
    if (extra) {  // the tile-major fill's further runs of ticket-heavy tiles, as tile_tickets_kernel lists them
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            const int64_t a = in_smem ? (int64_t)sT[t] : Tt[t], b = in_smem ? (int64_t)sT[t + 1] : Tt[t + 1];
            const int64_t runs = (b - a + ITEM_TICKETS - 1) / ITEM_TICKETS;
            if (runs > 1) {
                const int32_t pos = atomicAdd(&sum->n_extra, (int32_t)(runs - 1));
                for (int64_t k = 1; k < runs; ++k)
                    extra[pos + k - 1] = make_int2(t, (int32_t)k);
            }
        }
    }
    // fill work items: ceil(tickets / ITEM_TICKETS) per tile
    uint64_t items_total = 0;
    if (in_smem) {
        auto items_of = [&](int t) -> int32_t {
            return (int32_t)(((int64_t)sT[t + 1] - (int64_t)sT[t] + ITEM_TICKETS - 1) / ITEM_TICKETS);
        };
        uint64_t loc = 0;
        for (int t = s0; t < s1; ++t)
            loc += (uint64_t)items_of(t);
        int32_t off = (int32_t)block_excl_scan_u64(loc, red, &items_total);
        for (int t = s0; t < s1; ++t) {
            const int32_t cnt = items_of(t);
            item_off[t] = off;
            if (item_tile)
                for (int32_t k = 0; k < cnt; ++k)
                    item_tile[off + k] = t;
            off += cnt;
        }
    } else {
        for (int base = 0; base < T; base += blockDim.x) {
            const int t = base + threadIdx.x;
            const uint64_t cnt =
                (t < T) ? (uint64_t)((Tt[t + 1] - Tt[t] + ITEM_TICKETS - 1) / ITEM_TICKETS) : 0ull;
            uint64_t tot;
            const uint64_t ex = block_excl_scan_u64(cnt, red, &tot);
            if (t < T) {
                item_off[t] = (int32_t)(items_total + ex);
                if (item_tile)
                    for (uint64_t k = 0; k < cnt; ++k)
                        item_tile[items_total + ex + k] = t;
            }
            items_total += tot;
        }
    }
    if (threadIdx.x == 0) {
        item_off[T] = (int32_t)items_total;
        sum->n_items = (int32_t)items_total;
    }
    if (rpa) {
        for (int g = threadIdx.x; g <= G; g += blockDim.x) {
            const int64_t pos = goff[g];
            const uint64_t c = (pos >= N) ? Q : Ct[pos / TILE] + Cbl[g];
            Tg[g] = (pos >= N) ? N : tickets_below_grid(c, tg);
        }
    } else {
        // systematic keeps the group layout (the summary already holds its
        // extent, set whenever the layout changes); no routing
        if (threadIdx.x == 0) {
            sum->links = 0;
            sum->moved = 0;
        }
    }
}

// The tickets below every tile start and, for RPA and ARNA, every group
// start: one thread each, after tile_scan_kernel's prefix (the same counts
// tile_scan_kernel forms one block wide).  A tile with more than
// ITEM_TICKETS tickets lists its further runs (t, k), k >= 1, for the fill's
// extra blocks; the order of the list does not matter.
__global__ void __launch_bounds__(256) tile_tickets_kernel(
    int64_t N, int32_t T, const uint64_t *__restrict__ Ct, int64_t *__restrict__ Tt, DevSummary *__restrict__ sum,
    Divisor ndiv, const int64_t *__restrict__ goff, int32_t G, int rpa, const uint64_t *__restrict__ Cbl,
    int64_t *__restrict__ Tg, int2 *__restrict__ extra)
{
    if (sum->degenerate)
        return;  // kept by the N_eff test, or no usable weight
    const TicketGrid tg = ticket_grid(sum->Q, sum->u, sum->qN, sum->qR, ndiv);
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= T) {
        const int64_t a = (i == T) ? N : tickets_below_grid(Ct[i], tg);
        Tt[i] = a;
        if (i < T) {
            const int64_t b = (i + 1 == T) ? N : tickets_below_grid(Ct[i + 1], tg);
            const int64_t runs = (b - a + ITEM_TICKETS - 1) / ITEM_TICKETS;
            if (runs > 1) {
                const int32_t pos = atomicAdd(&sum->n_extra, (int32_t)(runs - 1));
                for (int64_t k = 1; k < runs; ++k)
                    extra[pos + k - 1] = make_int2(i, (int32_t)k);
            }
        }
    }
    if (rpa && i <= G) {
        const int64_t pos = goff[i];
        const uint64_t c = (pos >= N) ? sum->Q : Ct[pos / TILE] + Cbl[i];
        Tg[i] = (pos >= N) ? N : tickets_below_grid(c, tg);
    }
}

// ------------------------------------------------ kept tickets, GS and SGS
// GS and SGS leave every group at its balanced size n_g: a sender keeps n_g
// of its o_g tickets and sends the rest, a receiver keeps all o_g < n_g and
// is filled up.  The first keep_g = min(o_g, n_g) tickets of group g (tickets
// Tg[g] <= j < Tg[g+1], in ticket order) therefore land in slots off_g +
// (j - Tg[g]) of the balanced layout whatever the schedule pairs; the fill
// writes them there directly and only the sent tickets go to their ticket
// slot of anc_sys, for the routing copy of the links.
constexpr int KT_GROUPS = GT_MASKED + 1;  // groups holding one tile's particles, at most, for the table
struct KeptTable {
    int n;                         // groups in the table; -1: too many, look every ticket up
    int64_t start[KT_GROUPS + 1];  // first ticket of each group, then the end of the last one
    int64_t keep_end[KT_GROUPS];   // first ticket each group sends
    int64_t shift[KT_GROUPS];      // a kept ticket j goes to slot j + shift
};

// ticket_parents_contig with the kept / sent split: per staged chunk, every
// group's kept piece goes to anc (shifted to its balanced slot) and its sent
// piece to anc_sys + sent_shift, each as one store_staged run.  With kt.n < 0
// every ticket finds its group among Tg[0..G] by bisection (a tile crossed by
// more than KT_GROUPS groups).
__device__ __forceinline__ void ticket_parents_routed(const uint64_t *C, int n, uint64_t c0, const TicketGrid &tg,
                                                      int64_t j_lo, int64_t j_hi, uint16_t *stage,
                                                      const KeptTable &kt, int32_t *__restrict__ anc,
                                                      int32_t *__restrict__ anc_sys, int64_t sent_shift,
                                                      int32_t base, int64_t N, int32_t G, const Balanced &bl,
                                                      const int64_t *__restrict__ Tg, const int32_t *flags)
{
    for (int64_t c = j_lo; c < j_hi; c += STAGE_TICKETS) {
        const int64_t ce = (j_hi - c < STAGE_TICKETS) ? j_hi : c + STAGE_TICKETS;
        const int m = (int)(ce - c);
        ticket_parents(C, n, c0, tg, c, m, [&](int64_t j, int i) { stage[j - c] = (uint16_t)i; });
        __syncthreads();
        if (kt.n >= 0) {
            for (int e = 0; e < kt.n; ++e) {
                const int64_t a0 = c > kt.start[e] ? c : kt.start[e];
                const int64_t a1 = ce < kt.keep_end[e] ? ce : kt.keep_end[e];
                if (a0 < a1) {
                    if (a0 + kt.shift[e] >= 0 && a1 + kt.shift[e] <= N)
                        store_staged(anc + (a0 + kt.shift[e]), stage + (a0 - c), (int)(a1 - a0), base, n, flags);
                    else if (threadIdx.x == 0)
                        atomicOr(const_cast<int32_t *>(flags), FLAG_INTERNAL);  // inconsistent counts: never write out of bounds
                }
                const int64_t b0 = c > kt.keep_end[e] ? c : kt.keep_end[e];
                const int64_t b1 = ce < kt.start[e + 1] ? ce : kt.start[e + 1];
                if (b0 < b1) {
                    if (b0 + sent_shift >= 0 && b1 + sent_shift <= N)
                        store_staged(anc_sys + (b0 + sent_shift), stage + (b0 - c), (int)(b1 - b0), base, n,
                                     flags);
                    else if (threadIdx.x == 0)
                        atomicOr(const_cast<int32_t *>(flags), FLAG_INTERNAL);
                }
            }
        } else {
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                const int64_t j = c + k;
                int32_t a = 0, b = G - 1;  // the last g with Tg[g] <= j (Tg[0] = 0 <= j)
                while (a < b) {
                    const int32_t mid = (a + b + 1) >> 1;
                    if (__ldg(Tg + mid) <= j)
                        a = mid;
                    else
                        b = mid - 1;
                }
                const int64_t s0 = __ldg(Tg + a), o = __ldg(Tg + a + 1) - s0;
                const int64_t nk = target_of(bl, a);
                const int64_t keep = o < nk ? o : nk;
                const int64_t slot = (j - s0 < keep) ? balanced_offset(bl, a) + (j - s0) : j + sent_shift;
                int32_t *dst = (j - s0 < keep) ? anc : anc_sys;
                if (slot >= 0 && slot < N && PPF_DCHECK(stage[k] < n, flags, FLAG_INTERNAL))
                    dst[slot] = base + stage[k];
                else if (slot < 0 || slot >= N)
                    atomicOr(const_cast<int32_t *>(flags), FLAG_INTERNAL);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- R3 fill
// A fill block covers tickets [i_lo, i_hi) of one tile (at most
// ITEM_TICKETS); the tile's cumulative weights are built once in shared
// memory, the parents of the tickets are staged there and written out
// coalesced: to out[j] (systematic, LGS), or split into kept and sent
// tickets (GS, SGS: kr.anc set).  Dynamic shared memory: FILL_SMEM_BYTES.
struct KeptRoute {
    int32_t *anc;           // final ancestors; nullptr: every ticket to out[j]
    const int64_t *Tg;      // [G+1] tickets below each group start
    const int32_t *tile_g;  // [2T] per tile: first group starting at or after it, starts inside (capped)
    int32_t G;
    Balanced bl;            // the balanced layout GS and SGS leave
};

// The parents of tickets [i_lo, i_hi) of tile t: the tile's cumulative
// weights are built once in shared memory, the parents of the tickets are
// staged there and written out coalesced: to out[j] (systematic, LGS), or
// split into kept and sent tickets (GS, SGS: kr.anc set).
template <bool ROUTE>
__device__ __forceinline__ void fill_tile_tickets(const float *__restrict__ lw, int64_t N, Divisor ndiv,
                                                  const DevSummary *__restrict__ sum, uint64_t ct, int32_t t,
                                                  int64_t i_lo, int64_t i_hi, int32_t *__restrict__ out,
                                                  const KeptRoute &kr)
{
    extern __shared__ uint64_t fill_smem[];
    uint64_t *C = fill_smem;
    uint16_t *stage = reinterpret_cast<uint16_t *>(fill_smem + TILE_SMEM_U64);
    __shared__ uint64_t red[33];
    __shared__ KeptTable kt;
    const uint64_t sQ = sum->Q, su = sum->u, sqN = sum->qN;
    const uint32_t sqR = sum->qR;
    if (ROUTE && threadIdx.x >= blockDim.x - 32) {
        // the last warp: the groups holding the tile's particles, one lane
        // each (ga, the group of the tile's first particle, to gb, the last
        // group starting inside it)
        const int lane = threadIdx.x & 31;
        const int32_t gf = __ldg(kr.tile_g + 2 * t), ns = __ldg(kr.tile_g + 2 * t + 1);
        if (ns > GT_MASKED) {
            if (lane == 0)
                kt.n = -1;
        } else {
            const int32_t ga = gf > 0 ? gf - 1 : 0, gb = gf + ns - 1;  // gf = 0 only for tile 0, with ns >= 1
            const int ng = gb - ga + 1;
            if (lane <= ng) {
                const int32_t g = ga + lane;
                const int64_t s0 = __ldg(kr.Tg + g);
                kt.start[lane] = s0;
                if (lane < ng) {
                    const int64_t o = __ldg(kr.Tg + g + 1) - s0, nk = target_of(kr.bl, g);
                    kt.keep_end[lane] = s0 + (o < nk ? o : nk);
                    kt.shift[lane] = balanced_offset(kr.bl, g) - s0;
                }
            }
            if (lane == 0)
                kt.n = ng;
        }
    }
    const int64_t lo = (int64_t)t * TILE;
    const int n = (int)(N - lo < TILE ? N - lo : TILE);
    uint64_t q[TILE_ITEMS];
    tile_weights(lw, lo, n, sum->M, scale_bits(N), C, q);  // its barriers also publish the table
    tile_scan(q, C, red);
    const TicketGrid tg = ticket_grid(sQ, su, sqN, sqR, ndiv);
    if (ROUTE)
        ticket_parents_routed(C, n, ct, tg, i_lo, i_hi, stage, kt, kr.anc, out, 0, (int32_t)lo, N, kr.G, kr.bl,
                              kr.Tg, &sum->flags);
    else
        ticket_parents_contig(C, n, ct, tg, i_lo, i_hi, stage, out, (int32_t)lo, N, &sum->flags);
}

// The fill of the one-block tile scan (the allocation-free entry point): work
// item b covers tickets [i_lo, i_hi) of one tile (at most ITEM_TICKETS), the
// tile found from the item map, or by bisection over item_off without it.
// Dynamic shared memory: FILL_SMEM_BYTES.
__global__ void __launch_bounds__(TILE_THREADS) fill_kernel(
    const float *__restrict__ lw, int64_t N, int32_t T, Divisor ndiv, const DevSummary *__restrict__ sum,
    const uint64_t *__restrict__ Ct, const int64_t *__restrict__ Tt, const int32_t *__restrict__ item_off,
    const int32_t *__restrict__ item_tile, int32_t *__restrict__ out)
{
    __shared__ int32_t st;
    const int32_t b = blockIdx.x;
    // item_tile has an entry for every block of the launch: read it together
    // with the item count
    const int32_t t_pre = item_tile ? item_tile[b] : 0;
    if (b >= sum->n_items)
        return;
    if (item_tile == nullptr && threadIdx.x == 0) {
        int32_t a = 0, e = T;  // last t with item_off[t] <= b
        while (a < e) {
            const int32_t mid = (a + e + 1) >> 1;
            if (item_off[mid] <= b)
                a = mid;
            else
                e = mid - 1;
        }
        st = a;
    }
    if (item_tile == nullptr)
        __syncthreads();
    const int32_t t = item_tile ? t_pre : st;
    const int64_t tt0 = Tt[t], tt1 = Tt[t + 1];
    const int64_t i_lo = tt0 + (int64_t)(b - item_off[t]) * ITEM_TICKETS;
    const int64_t i_hi = (tt1 < i_lo + ITEM_TICKETS) ? tt1 : i_lo + ITEM_TICKETS;
    const KeptRoute none{nullptr, nullptr, nullptr, 0, Balanced{0, 0}};
    fill_tile_tickets<false>(lw, N, ndiv, sum, Ct[t], t, i_lo, i_hi, out, none);
}

// The fill after tile_tickets_kernel: block t < T takes tile t's first
// ITEM_TICKETS tickets, block T + e the e-th entry (t, k) of the list of
// further runs.  A tile without tickets returns at once.
template <bool ROUTE>
__global__ void __launch_bounds__(TILE_THREADS) fill_tiles_kernel(
    const float *__restrict__ lw, int64_t N, int32_t T, Divisor ndiv, const DevSummary *__restrict__ sum,
    const uint64_t *__restrict__ Ct, const int64_t *__restrict__ Tt, const int2 *__restrict__ extra,
    int32_t *__restrict__ out, KeptRoute kr)
{
    const int32_t b = blockIdx.x;
    if (sum->degenerate)
        return;  // kept by the N_eff test, or no usable weight
    int32_t t, k;
    if (b < T) {
        t = b;
        k = 0;
    } else {
        if (b - T >= sum->n_extra)
            return;
        const int2 e = extra[b - T];
        t = e.x;
        k = e.y;
    }
    const int64_t tt0 = Tt[t], tt1 = Tt[t + 1];
    const int64_t i_lo = tt0 + (int64_t)k * ITEM_TICKETS;
    const int64_t i_hi = (tt1 < i_lo + ITEM_TICKETS) ? tt1 : i_lo + ITEM_TICKETS;
    if (i_lo >= i_hi)
        return;  // a tile without tickets
    fill_tile_tickets<ROUTE>(lw, N, ndiv, sum, Ct[t], t, i_lo, i_hi, out, kr);
}

// ------------------------------------------------ two-stage RPA, stage 2
// Every group g draws its N_g = Tg[g+1] - Tg[g] offspring (stage 1: the
// global tickets of its cumulative range) again inside the group, by its own
// systematic draw over the same fixed-point weights with the offset from
// Philox(seed; g, frame, filter, GROUP).  They are written, in ticket order,
// where the global draw would have put them (ticket slots Tg[g] ..), so the
// RPA schedule and routing copy apply unchanged; with kept_anc set (GS, SGS)
// the group's first keep_g tickets go straight to its balanced slots in
// kept_anc instead, as in the one-stage fill.
//
// The group's total and the cumulative weight below any tile start inside it
// come from the global prefix of the tile pass (C(p) = Ct[p / TILE] + the
// local prefix at p; integer sums, so exactly the group's own sums), which
// lets a large group be split at tile boundaries: a group spanning more
// than GROUP_SPLIT particles is drawn by one block for its head (up to the
// first tile boundary) and one block per interior tile.  A smaller group
// with more than ITEM_TICKETS offspring is split by tickets instead: its
// block draws the first ITEM_TICKETS, and one more block each further run
// of ITEM_TICKETS, so that no block carries a heavy group alone.
constexpr int64_t GROUP_SPLIT = 2 * TILE;

// One thread per group: the group's draw; a large group lists all its tile
// parts (tile, g, run 0), a heavy small group its further runs (-1, g, r),
// r >= 1, in the split list (four ints an entry; the order of the list does
// not matter: every entry writes its own tickets).
__global__ void __launch_bounds__(256) group_grid_kernel(
    int64_t N, int32_t G, const int64_t *__restrict__ goff, const int64_t *__restrict__ Tg,
    const uint64_t *__restrict__ Ct, const uint64_t *__restrict__ Cbl, DevSummary *__restrict__ sum, double ess_thr,
    uint64_t seed, uint32_t fid, uint32_t frame, GroupGrid *__restrict__ grid, int4 *__restrict__ split,
    Balanced bl)
{
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G || kept_by_ess(sum, ess_thr) || sum->degenerate)
        return;
    const uint64_t Q = sum->Q;
    const int64_t a = goff[g], e = goff[g + 1];
    const uint64_t ca = (a >= N) ? Q : Ct[a / TILE] + Cbl[g];
    const uint64_t ce = (e >= N) ? Q : Ct[e / TILE] + Cbl[g + 1];
    const int64_t nt = Tg[g + 1] - Tg[g];
    GroupGrid gg;
    gg.Ca = ca;
    gg.Q = ce - ca;
    gg.nt = (nt > 0 && gg.Q > 0) ? (uint32_t)nt : 0u;
    gg.u = gg.qN = gg.dm = 0;
    gg.qR = 0;
    gg.p0 = a;
    gg.p1 = e;
    gg.tg0 = Tg[g];
    {
        const int64_t nk = target_of(bl, g);
        gg.keep = nt < nk ? nt : nk;
        gg.shift = balanced_offset(bl, g);
    }
    if (gg.nt > 0) {
        gg.u = ticket_offset(seed, fid, frame, PURPOSE_GROUP, (uint32_t)g, gg.Q);
        gg.dm = make_divisor(gg.nt).m;
        gg.qN = gg.Q / gg.nt;
        gg.qR = (uint32_t)(gg.Q % gg.nt);
    }
    grid[g] = gg;
    if (gg.nt == 0)
        return;
    if (e - a > GROUP_SPLIT) {
        const int64_t t1 = a / TILE, t2 = (e - 1) / TILE;  // every tile the group reaches
        const int32_t pos = atomicAdd(&sum->n_split, (int32_t)(t2 - t1 + 1));
        for (int64_t t = t1; t <= t2; ++t)
            split[pos + (t - t1)] = make_int4((int32_t)t, g, 0, 0);
    } else if (nt > ITEM_TICKETS) {
        const int32_t runs = (int32_t)((nt + ITEM_TICKETS - 1) / ITEM_TICKETS);
        const int32_t pos = atomicAdd(&sum->n_split, runs - 1);
        for (int32_t r = 1; r < runs; ++r)
            split[pos + r - 1] = make_int4(-1, g, r, 0);
    }
}

// The part of a large group in one tile: its particles and the group's
// cumulative weight below them.
__device__ __forceinline__ void tile_part(const GroupGrid &gg, int32_t t, const uint64_t *__restrict__ Ct,
                                          int64_t &p0, int64_t &p1, uint64_t &carry)
{
    const int64_t lo = (int64_t)t * TILE;
    p0 = lo > gg.p0 ? lo : gg.p0;
    p1 = lo + TILE < gg.p1 ? lo + TILE : gg.p1;
    carry = p0 == gg.p0 ? 0ull : Ct[t] - gg.Ca;
}

// One thread per tile part listed by group_grid_kernel: a part with more than
// ITEM_TICKETS offspring appends its further runs (tile, g, r), r >= 1, so
// that a heavy tile of a large group is drawn by several blocks too.
__global__ void __launch_bounds__(256) split_runs_kernel(const uint64_t *__restrict__ Ct,
                                                         const GroupGrid *__restrict__ grid, int4 *__restrict__ split,
                                                         DevSummary *__restrict__ sum, double ess_thr)
{
    if (kept_by_ess(sum, ess_thr) || sum->degenerate)
        return;
    const int32_t n0 = sum->n_split;  // the entries group_grid_kernel listed; the runs go after them
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += gridDim.x * blockDim.x) {
        const int4 en = split[i];
        if (en.x < 0 || en.z != 0)
            continue;
        const GroupGrid gg = grid[en.y];
        int64_t p0, p1;
        uint64_t c_lo;
        tile_part(gg, en.x, Ct, p0, p1, c_lo);
        const uint64_t c_hi = p1 == gg.p1 ? gg.Q : Ct[en.x + 1] - gg.Ca;
        const int64_t nt = gg.nt;
        const int64_t j_lo = c_lo == 0 ? 0 : tickets_below(c_lo, nt, gg.u, gg.Q);
        const int64_t j_hi = c_hi == gg.Q ? nt : tickets_below(c_hi, nt, gg.u, gg.Q);
        if (j_hi - j_lo > ITEM_TICKETS) {
            const int32_t runs = (int32_t)((j_hi - j_lo + ITEM_TICKETS - 1) / ITEM_TICKETS);
            const int32_t pos = n0 + atomicAdd(&sum->n_runs, runs - 1);
            for (int32_t r = 1; r < runs; ++r)
                split[pos + r - 1] = make_int4(en.x, en.y, r, 0);
        }
    }
}

// One work item of the two-stage draw: particles [p0, p1) of group gg, carry
// the group's cumulative weight below p0.  Its tickets: the group's [j0, j1)
// among them (run < 0), or run `run` of ITEM_TICKETS among the tickets of a
// one-tile part (run >= 0).
__device__ __forceinline__ void group_fill_item(const float *__restrict__ lw, int64_t N, int32_t G,
                                                const int64_t *__restrict__ Tg, const GroupGrid &gg, int64_t p0,
                                                int64_t p1, int64_t j0, int64_t j1, int32_t run, uint64_t carry,
                                                float M, int s, const DevSummary *__restrict__ sum,
                                                int32_t *__restrict__ out, int32_t *__restrict__ kept_anc,
                                                const Balanced &bl, uint64_t *C, uint16_t *stage, uint64_t *red)
{
    const int64_t nt = gg.nt;
    Divisor dv;
    dv.m = gg.dm;
    dv.d = gg.nt;
    const TicketGrid tg = ticket_grid(gg.Q, gg.u, gg.qN, gg.qR, dv);
    KeptTable kt;  // one group, in local ticket numbers
    kt.n = 1;
    kt.start[0] = 0;
    kt.start[1] = nt;
    kt.keep_end[0] = gg.keep;
    kt.shift[0] = gg.shift;
    // chunks of at most TILE particles; the local tickets of a chunk with
    // cumulative weight [carry, carry + total) inside the group are
    // [T(carry), T(carry + total)), T the count below of the nt tickets
    for (int64_t c0 = p0; c0 < p1; c0 += TILE) {
        const int n = (int)(p1 - c0 < TILE ? p1 - c0 : TILE);
        uint64_t q[TILE_ITEMS];
        tile_weights(lw, c0, n, M, s, C, q);
        const uint64_t tot = tile_scan(q, C, red);
        // no ticket lies below the group's start, all of them below its end
        const int64_t c_lo = carry == 0 ? 0 : tickets_below(carry, nt, gg.u, gg.Q);
        const int64_t c_hi = c0 + n == gg.p1 ? nt : tickets_below(carry + tot, nt, gg.u, gg.Q);
        int64_t t_lo, t_hi;
        if (run >= 0) {
            t_lo = c_lo + (int64_t)run * ITEM_TICKETS;
            t_hi = (t_lo + ITEM_TICKETS < c_hi) ? t_lo + ITEM_TICKETS : c_hi;
        } else {
            t_lo = c_lo > j0 ? c_lo : j0;
            t_hi = c_hi < j1 ? c_hi : j1;
        }
        if (kept_anc)
            ticket_parents_routed(C, n, carry, tg, t_lo, t_hi, stage, kt, kept_anc, out, gg.tg0, (int32_t)c0, N, G,
                                  bl, Tg, &sum->flags);
        else
            ticket_parents_contig(C, n, carry, tg, t_lo, t_hi, stage, out + gg.tg0, (int32_t)c0,
                                  (nt < N - gg.tg0) ? nt : N - gg.tg0, &sum->flags);
        carry += tot;
        __syncthreads();
    }
}

// Blocks [0, n_workers) take the split list's entries in turn; block
// n_workers + g takes a small group g whole, or its first ITEM_TICKETS
// tickets when it is heavy (a large group is all in the split list).
// s: scale_bits(N).
__global__ void __launch_bounds__(TILE_THREADS, 4) group_fill_kernel(
    const float *__restrict__ lw, int64_t N, int32_t G, const int64_t *__restrict__ Tg,
    const uint64_t *__restrict__ Ct, const GroupGrid *__restrict__ grid, const int4 *__restrict__ split,
    int32_t n_workers, const DevSummary *__restrict__ sum, double ess_thr, int32_t *__restrict__ out,
    int32_t *__restrict__ kept_anc, Balanced bl, int s)
{
    extern __shared__ uint64_t fill_smem[];  // FILL_SMEM_BYTES
    uint64_t *C = fill_smem;
    uint16_t *stage = reinterpret_cast<uint16_t *>(fill_smem + TILE_SMEM_U64);
    __shared__ uint64_t red[33];
    if ((int32_t)blockIdx.x >= n_workers) {  // a group block: one item, no loop
        const GroupGrid gg = grid[blockIdx.x - n_workers];
        const double ess = sum->ess;
        const int32_t deg = sum->degenerate;
        const float M = sum->M;
        if (ess >= ess_thr || deg || gg.nt == 0 || gg.p1 - gg.p0 > GROUP_SPLIT)
            return;  // kept by the N_eff test, no usable weight, no offspring, or a large group
        const int64_t j1 = gg.nt > ITEM_TICKETS ? ITEM_TICKETS : gg.nt;  // a heavy group's first run
        group_fill_item(lw, N, G, Tg, gg, gg.p0, gg.p1, 0, j1, -1, 0, M, s, sum, out, kept_anc, bl, C, stage,
                        red);
        return;
    }
    if (sum->ess >= ess_thr || sum->degenerate)
        return;
    const float M = sum->M;
    const int32_t n_items = sum->n_split + sum->n_runs;
    for (int32_t it = (int32_t)blockIdx.x; it < n_items; it += n_workers) {
        const int4 en = split[it];
        const GroupGrid gg = grid[en.y];
        if (en.x >= 0) {  // run en.z of a large group's part in tile en.x
            int64_t p0, p1;
            uint64_t carry;
            tile_part(gg, en.x, Ct, p0, p1, carry);
            group_fill_item(lw, N, G, Tg, gg, p0, p1, 0, 0, en.z, carry, M, s, sum, out, kept_anc, bl, C, stage,
                            red);
        } else {  // run en.z of a heavy small group
            const int64_t j0 = (int64_t)en.z * ITEM_TICKETS;
            const int64_t j1 = (j0 + ITEM_TICKETS < (int64_t)gg.nt) ? j0 + ITEM_TICKETS : (int64_t)gg.nt;
            group_fill_item(lw, N, G, Tg, gg, gg.p0, gg.p1, j0, j1, -1, 0, M, s, sum, out, kept_anc, bl, C, stage,
                            red);
        }
    }
}

// ------------------------------------------------------------ RPA schedule
// One block.  Senders / receivers from the offspring counts o_g = T_{g+1} -
// T_g and the balanced targets n_g; SGS and LGS sort both lists by amount,
// descending, ties by group index (a merge sort in shared memory).  GS/SGS
// links are the pieces of [0, D) cut at every sender and receiver prefix
// boundary (D = total surplus = total deficit); LGS pairs the i-th sender
// with the i-th receiver.  Output: new group offsets and the routing
// segments (ticket start, slot start, length) with their copy work items
// (GS and SGS: the links only, from schedule_links_balanced).
struct SchedArgs {
    int64_t N;
    int32_t G;
    int scheme;
    const int64_t *goff;
    int64_t *goff_new;
    const int64_t *Tg;
    uint64_t *key;      // [2 * G]  (sender keys, receiver keys)
    int64_t *val;       // [5 * G]  (PS, PR, sent, recv, merge buffer)
    int32_t *seg_chunk; // [2G + 2]
    int64_t *seg_tick, *seg_dst, *seg_len;  // [2G + 1]
    DevSummary *sum;
    int links_only;  // the fill wrote the kept segments already: copy work items for the links only
    Balanced bl;     // the balanced targets n_g
};

// block-wide exclusive scan of an int64 array in place (single block)
__device__ void block_scan_i64(int64_t *a, int n, uint64_t *red, int64_t *total_out)
{
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    uint64_t s = 0;
    for (int k = 0; k < per; ++k)
        if (i0 + k < n)
            s += (uint64_t)a[i0 + k];
    uint64_t total;
    uint64_t run = block_excl_scan_u64(s, red, &total);
    __syncthreads();
    for (int k = 0; k < per; ++k)
        if (i0 + k < n) {
            const int64_t v = a[i0 + k];
            a[i0 + k] = (int64_t)run;
            run += (uint64_t)v;
        }
    if (total_out)
        *total_out = (int64_t)total;
    __syncthreads();
}

// Sort (ascending) of n <= cap distinct u64 keys, one block of 1024 threads.
// sm: cap keys, then two index buffers of cap u16 (sort_smem_bytes(cap) in
// all, cap <= MAX_SCHED_GROUPS); g may be sm itself.  A merge sort on
// indices: every thread sorts a run of 16 in registers, then the merge
// levels, each thread writing 16 outputs after a merge-path search of its
// diagonal.  Launches size the buffer by their G, not by the largest G, so
// that the rest of the SM's 256 KB stays L1 cache for the kernel's global
// reads.
constexpr int SORT_PER = 16;
// every key needs a thread: the 1024 threads' runs cover the largest group count
static_assert(SORT_PER * 1024 >= MAX_SCHED_GROUPS, "block_sort_u64 covers at most SORT_PER x 1024 keys");
constexpr size_t SORT_SMEM_BYTES = (sizeof(uint64_t) + 2 * sizeof(uint16_t)) * MAX_SCHED_GROUPS;
__host__ __device__ inline size_t sort_smem_bytes(int cap)
{
    return (sizeof(uint64_t) + 2 * sizeof(uint16_t)) * (size_t)(cap > 0 ? cap : 1);
}

__device__ void block_sort_u64(uint64_t *g, int n, uint64_t *sm, int cap)
{
    uint16_t *ia = reinterpret_cast<uint16_t *>(sm + cap), *ib = ia + cap;
    if (g != sm)
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            sm[i] = g[i];
    __syncthreads();
    const int t0 = threadIdx.x * SORT_PER;
    {
        uint64_t k[SORT_PER];
        uint16_t id[SORT_PER];
#pragma unroll
        for (int e = 0; e < SORT_PER; ++e) {
            k[e] = (t0 + e < n) ? sm[t0 + e] : ~0ull;  // past the end: sorts last
            id[e] = (uint16_t)(t0 + e);
        }
#pragma unroll
        for (int e = 1; e < SORT_PER; ++e)
#pragma unroll
            for (int f = e; f > 0; --f)
                if (k[f] < k[f - 1]) {
                    const uint64_t tk = k[f];
                    k[f] = k[f - 1];
                    k[f - 1] = tk;
                    const uint16_t ti = id[f];
                    id[f] = id[f - 1];
                    id[f - 1] = ti;
                }
#pragma unroll
        for (int e = 0; e < SORT_PER; ++e)
            if (t0 + e < n)
                ia[t0 + e] = id[e];
    }
    __syncthreads();
    uint16_t *src = ia, *dst = ib;
    for (int w = SORT_PER; w < n; w *= 2) {
        if (t0 < n) {
            const int base = (t0 / (2 * w)) * (2 * w);
            const int an = (n - base < w) ? n - base : w;
            const int b0 = base + w;
            const int bn = (n - b0 <= 0) ? 0 : ((n - b0 < w) ? n - b0 : w);
            const int d = t0 - base;
            int lo = d - bn > 0 ? d - bn : 0, hi = d < an ? d : an;
            while (lo < hi) {  // merge path: i taken from the first run, d - i from the second
                const int mid = (lo + hi) >> 1;
                if (sm[src[base + mid]] < sm[src[b0 + d - mid - 1]])
                    lo = mid + 1;
                else
                    hi = mid;
            }
            int i = lo, j = d - lo;
            const int cnt = (an + bn - d < SORT_PER) ? an + bn - d : SORT_PER;
            for (int e = 0; e < cnt; ++e) {
                const bool take_a = i < an && (j >= bn || sm[src[base + i]] < sm[src[b0 + j]]);
                dst[t0 + e] = take_a ? src[base + i] : src[b0 + j];
                i += take_a ? 1 : 0;
                j += take_a ? 0 : 1;
            }
        }
        __syncthreads();
        uint16_t *t = src;
        src = dst;
        dst = t;
    }
    uint64_t k[SORT_PER];
#pragma unroll
    for (int e = 0; e < SORT_PER; ++e)
        k[e] = (t0 + e < n) ? sm[src[t0 + e]] : 0ull;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < SORT_PER; ++e)
        if (t0 + e < n)
            g[t0 + e] = k[e];
    __syncthreads();
}

// first index in sorted a[0..n) with a[i] > v
__device__ __forceinline__ int upper_bound_i64(const int64_t *a, int n, int64_t v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] > v)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int lower_bound_i64(const int64_t *a, int n, int64_t v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// first index in sorted a[0..n) with a[i] > v (int32 values in shared memory)
__device__ __forceinline__ int upper_bound_i32(const int32_t *a, int n, int32_t v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] > v)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int n, int32_t v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// exclusive prefix of a[0..n) in place, a[n] = the total (one block; every
// thread takes one contiguous segment)
__device__ void block_scan_smem_i32(int32_t *a, int n, uint64_t *red)
{
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    uint64_t loc = 0;
    for (int k = 0; k < per; ++k)
        if (i0 + k < n)
            loc += (uint32_t)a[i0 + k];
    uint64_t total;
    uint64_t run = block_excl_scan_u64(loc, red, &total);
    for (int k = 0; k < per; ++k)
        if (i0 + k < n) {
            const int32_t v = a[i0 + k];
            a[i0 + k] = (int32_t)run;
            run += (uint32_t)v;
        }
    if (threadIdx.x == 0)
        a[n] = (int32_t)total;
    __syncthreads();
}

// Shared memory of schedule_kernel: the sort's buffer, and at least what
// schedule_links_balanced lays out (two u16 id lists, three int32 arrays).
__host__ __device__ inline size_t sched_smem_bytes(int G)
{
    const size_t need = 10 * (size_t)(G > 0 ? G : 1) + 64;
    const size_t sort = sort_smem_bytes(G);
    return sort > need ? sort : need;
}

// GS and SGS: every group ends at its balanced size, so the new offsets are
// the balanced ones and every sender keeps exactly n_g of its tickets (the
// fill already wrote those).  What remains are the links: the pieces of
// [0, D) cut at every sender and receiver prefix boundary, in the senders'
// and receivers' list order (group order for GS, sorted for SGS), and the
// copy work items of the links.  Everything but Tg stays in shared memory:
// the list order's group ids (u16), the prefix sums of the amounts (int32,
// with the total D as a sentinel), and the merge of the two prefix lists.
__device__ void schedule_links_balanced(const SchedArgs &A, int nS, int nR, bool sorted, uint64_t *sm,
                                        uint64_t *red)
{
    const int32_t G = A.G;
    const Balanced &bl = A.bl;
    DevSummary *sum = A.sum;
    const uint64_t *Skey = A.key, *Rkey = A.key + G;
    uint16_t *gS = reinterpret_cast<uint16_t *>(sm);
    uint16_t *gR = gS + nS;
    int32_t *PS = reinterpret_cast<int32_t *>(sm) + ((nS + nR + 1) / 2 + 1);  // after the ids, 4-byte aligned
    int32_t *PR = PS + nS + 1;
    int32_t *MG = PR + nR + 1;
    auto amount = [&](uint64_t k) -> int32_t {
        return sorted ? (int32_t)(0xFFFFFFFFFFull - (k >> 24)) : (int32_t)(k >> 24);
    };
    // 1. ids and amounts in list order; the balanced offsets and extent
    for (int i = threadIdx.x; i < nS; i += blockDim.x) {
        const uint64_t k = Skey[i];
        gS[i] = (uint16_t)(k & 0xFFFFFFull);
        PS[i] = amount(k);
    }
    for (int j = threadIdx.x; j < nR; j += blockDim.x) {
        const uint64_t k = Rkey[j];
        gR[j] = (uint16_t)(k & 0xFFFFFFull);
        PR[j] = amount(k);
    }
    for (int g = threadIdx.x; g <= G; g += blockDim.x)
        A.goff_new[g] = balanced_offset(bl, g);
    if (threadIdx.x == 0) {
        sum->max_group = bl.q + (bl.r > 0 ? 1 : 0);
        sum->min_group = bl.q;
    }
    __syncthreads();
    // 2. exclusive prefix sums (PS[nS] = PR[nR] = D)
    block_scan_smem_i32(PS, nS, red);
    block_scan_smem_i32(PR, nR, red);
    // 3. the merge of the two start lists (senders first on ties)
    for (int i = threadIdx.x; i < nS; i += blockDim.x)
        MG[i + lower_bound_i32(PR, nR, PS[i])] = PS[i];
    for (int j = threadIdx.x; j < nR; j += blockDim.x)
        MG[j + upper_bound_i32(PS, nS, PR[j])] = PR[j];
    __syncthreads();
    // 4. one link per distinct start, in order; each thread takes one
    //    contiguous range of the merge and knows its links' places
    const int nm = nS + nR;
    const int per = (nm + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    uint64_t c = 0;
    for (int k = 0; k < per; ++k) {
        const int i = i0 + k;
        if (i < nm && (i == 0 || MG[i] != MG[i - 1]))
            ++c;
    }
    uint64_t L;
    const uint64_t pos0 = block_excl_scan_u64(c, red, &L);
    uint64_t pos = pos0, chunks = 0;
    for (int k = 0; k < per; ++k) {
        const int i = i0 + k;
        if (i < nm && (i == 0 || MG[i] != MG[i - 1])) {
            const int32_t a = MG[i];
            const int si = upper_bound_i32(PS, nS, a) - 1;  // the sender piece holding a
            const int rj = upper_bound_i32(PR, nR, a) - 1;
            const int32_t e = PS[si + 1] < PR[rj + 1] ? PS[si + 1] : PR[rj + 1];
            const int32_t gs = gS[si], gr = gR[rj];
            const int64_t ts = A.Tg[gs], tr0 = A.Tg[gr], tr1 = A.Tg[gr + 1];
            // a sender keeps n_s; a receiver keeps its o_r and is filled after them
            A.seg_tick[G + pos] = ts + target_of(bl, gs) + (a - PS[si]);
            A.seg_dst[G + pos] = balanced_offset(bl, gr) + (tr1 - tr0) + (a - PR[rj]);
            A.seg_len[G + pos] = e - a;
            chunks += (uint64_t)((e - a + COPY_CHUNK - 1) / COPY_CHUNK);
            ++pos;
        }
    }
    // 5. copy work items: none for the kept segments [0, G), then the links
    uint64_t total_chunks;
    uint64_t run = block_excl_scan_u64(chunks, red, &total_chunks);
    for (int g = threadIdx.x; g < G; g += blockDim.x)
        A.seg_chunk[g] = 0;
    for (uint64_t p = pos0; p < pos; ++p) {
        A.seg_chunk[G + p] = (int32_t)run;
        run += (uint64_t)((A.seg_len[G + p] + COPY_CHUNK - 1) / COPY_CHUNK);
    }
    if (threadIdx.x == 0) {
        const int32_t nseg = G + (int32_t)L;
        A.seg_chunk[nseg] = (int32_t)total_chunks;
        A.seg_chunk[2 * G + 1] = nseg;  // the segment count
        sum->n_chunks = (int32_t)total_chunks;
        sum->links = (int64_t)L;
        sum->moved = PS[nS];
    }
}

__global__ void __launch_bounds__(1024) schedule_kernel(SchedArgs A)
{
    extern __shared__ uint64_t sm[];   // sort_smem_bytes(G) (GS: G words)
    __shared__ uint64_t red[33];
    __shared__ int nS_s, nR_s, L_s;
    const int32_t G = A.G;
    DevSummary *sum = A.sum;
    if (sum->degenerate) {
        for (int g = threadIdx.x; g <= G; g += blockDim.x)
            A.goff_new[g] = A.goff[g];
        if (threadIdx.x == 0) {
            sum->n_chunks = 0;
            sum->links = 0;
            sum->moved = 0;
        }
        return;
    }
    uint64_t *Skey = A.key, *Rkey = A.key + G;
    int64_t *PS = A.val, *PR = A.val + G;
    // 1. senders / receivers, compacted in group order.  key = amount << 24 | g
    //    (amount <= N < 2^31 fits 40 bits; g < 2^24).  For sorting by amount
    //    descending then g ascending we sort ((2^40-1-amount) << 24 | g).
    if (threadIdx.x == 0) {
        nS_s = 0;
        nR_s = 0;
    }
    __syncthreads();
    // stable compaction via block scan of flags over contiguous per-thread ranges
    {
        const int per = (G + blockDim.x - 1) / blockDim.x;
        const int g0 = threadIdx.x * per;
        uint64_t cs = 0, cr = 0;
        for (int k = 0; k < per; ++k) {
            const int g = g0 + k;
            if (g < G) {
                const int64_t o = A.Tg[g + 1] - A.Tg[g], t = target_of(A.bl, g);
                cs += (o > t);
                cr += (o < t);
            }
        }
        uint64_t ts, tr;
        uint64_t ps = block_excl_scan_u64(cs, red, &ts);
        uint64_t pr = block_excl_scan_u64(cr, red, &tr);
        const bool sorted = (A.scheme != PPF_RPA_GS);
        for (int k = 0; k < per; ++k) {
            const int g = g0 + k;
            if (g < G) {
                const int64_t o = A.Tg[g + 1] - A.Tg[g], t = target_of(A.bl, g);
                if (o > t) {
                    const uint64_t amt = (uint64_t)(o - t);
                    Skey[ps++] = sorted ? (((0xFFFFFFFFFFull - amt) << 24) | (uint64_t)g) : ((amt << 24) | (uint64_t)g);
                }
                if (o < t) {
                    const uint64_t amt = (uint64_t)(t - o);
                    Rkey[pr++] = sorted ? (((0xFFFFFFFFFFull - amt) << 24) | (uint64_t)g) : ((amt << 24) | (uint64_t)g);
                }
            }
        }
        if (threadIdx.x == 0) {
            nS_s = (int)ts;
            nR_s = (int)tr;
        }
    }
    __syncthreads();
    const int nS = nS_s, nR = nR_s;
    const bool sorted = (A.scheme != PPF_RPA_GS);
    if (sorted) {
        block_sort_u64(Skey, nS, sm, G);
        block_sort_u64(Rkey, nR, sm, G);
    }
    if (A.links_only) {
        schedule_links_balanced(A, nS, nR, sorted, sm, red);
        return;
    }
    auto amount = [&](uint64_t k) -> int64_t {
        return sorted ? (int64_t)(0xFFFFFFFFFFull - (k >> 24)) : (int64_t)(k >> 24);
    };
    auto group = [&](uint64_t k) -> int32_t { return (int32_t)(k & 0xFFFFFFull); };
    // per-group sent / received totals
    int64_t *sent = A.val + 2 * G, *recv = A.val + 3 * G;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        sent[g] = 0;
        recv[g] = 0;
    }
    __syncthreads();
    int L = 0;
    if (A.scheme == PPF_RPA_LGS) {
        L = nS < nR ? nS : nR;
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const int64_t a = amount(Skey[i]), b = amount(Rkey[i]);
            const int64_t c = a < b ? a : b;
            sent[group(Skey[i])] = c;
            recv[group(Rkey[i])] = c;
        }
    } else {
        for (int i = threadIdx.x; i < nS; i += blockDim.x)
            sent[group(Skey[i])] = amount(Skey[i]);
        for (int i = threadIdx.x; i < nR; i += blockDim.x)
            recv[group(Rkey[i])] = amount(Rkey[i]);
    }
    __syncthreads();
    // 2. new sizes and offsets: m'_g = o_g - sent_g + recv_g
    int64_t *off = A.goff_new;
    for (int g = threadIdx.x; g < G; g += blockDim.x)
        off[g] = (A.Tg[g + 1] - A.Tg[g]) - sent[g] + recv[g];
    __syncthreads();
    {
        int64_t mx = 0, mn = INT64_MAX;
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            mx = off[g] > mx ? off[g] : mx;
            mn = off[g] < mn ? off[g] : mn;
        }
        __shared__ long long smx[32], smn[32];
        for (int o = 16; o > 0; o >>= 1) {
            const long long a = __shfl_xor_sync(0xffffffffu, (long long)mx, o);
            const long long b = __shfl_xor_sync(0xffffffffu, (long long)mn, o);
            mx = a > mx ? a : mx;
            mn = b < mn ? b : mn;
        }
        if ((threadIdx.x & 31) == 0) {
            smx[threadIdx.x >> 5] = mx;
            smn[threadIdx.x >> 5] = mn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long a = 0, b = INT64_MAX;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                a = smx[w] > a ? smx[w] : a;
                b = smn[w] < b ? smn[w] : b;
            }
            sum->max_group = a;
            sum->min_group = b;
        }
        __syncthreads();
    }
    int64_t tot;
    block_scan_i64(off, G, red, &tot);
    if (threadIdx.x == 0)
        off[G] = tot;
    __syncthreads();
    // 3. kept segments: group g keeps its first o_g - sent_g tickets
    int64_t *seg_len = A.seg_len, *seg_tick = A.seg_tick, *seg_dst = A.seg_dst;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        seg_tick[g] = A.Tg[g];
        seg_dst[g] = off[g];
        seg_len[g] = (A.Tg[g + 1] - A.Tg[g]) - sent[g];
    }
    // 4. links
    if (A.scheme == PPF_RPA_LGS) {
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const int32_t s = group(Skey[i]), r = group(Rkey[i]);
            const int64_t c = sent[s];
            const int64_t keep_s = (A.Tg[s + 1] - A.Tg[s]) - c;
            const int64_t keep_r = A.Tg[r + 1] - A.Tg[r];
            seg_tick[G + i] = A.Tg[s] + keep_s;
            seg_dst[G + i] = off[r] + keep_r;
            seg_len[G + i] = c;
        }
        if (threadIdx.x == 0)
            L_s = L;
        __syncthreads();
    } else {
        // prefix sums of the amounts in list order (inclusive)
        for (int i = threadIdx.x; i < nS; i += blockDim.x)
            PS[i] = amount(Skey[i]);
        for (int i = threadIdx.x; i < nR; i += blockDim.x)
            PR[i] = amount(Rkey[i]);
        __syncthreads();
        int64_t d1, d2;
        block_scan_i64(PS, nS, red, &d1);
        block_scan_i64(PR, nR, red, &d2);
        // now PS[i], PR[j] are exclusive starts; piece starts are the union of
        // both start sets (0 is in both).  Merge them (PS first on ties).
        int64_t *MG = A.val + 4 * G;  // at most nS + nR <= G entries
        // the binary searches below run on shared copies of the two prefix
        // arrays (nS + nR <= G <= MAX_SCHED_GROUPS entries; the sort is done)
        int64_t *sPS = reinterpret_cast<int64_t *>(sm), *sPR = sPS + nS;
        __syncthreads();
        for (int i = threadIdx.x; i < nS; i += blockDim.x)
            sPS[i] = PS[i];
        for (int j = threadIdx.x; j < nR; j += blockDim.x)
            sPR[j] = PR[j];
        __syncthreads();
        for (int i = threadIdx.x; i < nS; i += blockDim.x)
            MG[i + lower_bound_i64(sPR, nR, sPS[i])] = sPS[i];
        for (int j = threadIdx.x; j < nR; j += blockDim.x)
            MG[j + upper_bound_i64(sPS, nS, sPR[j])] = sPR[j];
        __syncthreads();
        const int nm = nS + nR;
        // distinct starts -> links; store compacted into seg arrays after G
        {
            const int per = (nm + blockDim.x - 1) / blockDim.x;
            const int i0 = threadIdx.x * per;
            uint64_t c = 0;
            for (int k = 0; k < per; ++k) {
                const int i = i0 + k;
                if (i < nm && (i == 0 || MG[i] != MG[i - 1]))
                    ++c;
            }
            uint64_t tl;
            uint64_t pos = block_excl_scan_u64(c, red, &tl);
            for (int k = 0; k < per; ++k) {
                const int i = i0 + k;
                if (i < nm && (i == 0 || MG[i] != MG[i - 1])) {
                    const int64_t a = MG[i];
                    const int si = upper_bound_i64(sPS, nS, a) - 1;  // sender piece contains a
                    const int rj = upper_bound_i64(sPR, nR, a) - 1;
                    const int64_t se = sPS[si] + amount(Skey[si]);
                    const int64_t re = sPR[rj] + amount(Rkey[rj]);
                    const int64_t e = se < re ? se : re;
                    const int32_t s = group(Skey[si]), r = group(Rkey[rj]);
                    const int64_t keep_s = (A.Tg[s + 1] - A.Tg[s]) - sent[s];
                    const int64_t keep_r = A.Tg[r + 1] - A.Tg[r];
                    seg_tick[G + pos] = A.Tg[s] + keep_s + (a - sPS[si]);
                    seg_dst[G + pos] = off[r] + keep_r + (a - sPR[rj]);
                    seg_len[G + pos] = e - a;
                    ++pos;
                }
            }
            if (threadIdx.x == 0)
                L_s = (nm > 0) ? (int)tl : 0;
        }
        __syncthreads();
    }
    L = L_s;
    const int nseg = G + L;
    // 5. copy work items per segment
    {
        const int per = (nseg + blockDim.x - 1) / blockDim.x;
        const int i0 = threadIdx.x * per;
        uint64_t c = 0, mv = 0;
        for (int k = 0; k < per; ++k) {
            const int i = i0 + k;
            if (i < nseg) {
                if (i >= G || !A.links_only)
                    c += (uint64_t)((seg_len[i] + COPY_CHUNK - 1) / COPY_CHUNK);
                if (i >= G)
                    mv += (uint64_t)seg_len[i];
            }
        }
        uint64_t tc, tmv;
        uint64_t run = block_excl_scan_u64(c, red, &tc);
        block_excl_scan_u64(mv, red, &tmv);
        for (int k = 0; k < per; ++k) {
            const int i = i0 + k;
            if (i < nseg) {
                A.seg_chunk[i] = (int32_t)run;
                if (i >= G || !A.links_only)
                    run += (uint64_t)((seg_len[i] + COPY_CHUNK - 1) / COPY_CHUNK);
            }
        }
        if (threadIdx.x == 0) {
            A.seg_chunk[nseg] = (int32_t)tc;
            sum->n_chunks = (int32_t)tc;
            sum->links = L;
            sum->moved = (int64_t)tmv;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        A.seg_chunk[2 * G + 1] = nseg;  // remember the segment count
}

// routing copy: anc[dst + k] = anc_sys[tick + k] for every segment, in work
// items of COPY_CHUNK slots; blocks loop over the items.  The first warp finds
// an item's segment (the last with seg_chunk <= b) by a 32-way search: each
// round probes 32 evenly spaced entries at once, so about three dependent
// loads locate it among tens of thousands of segments.
__global__ void __launch_bounds__(256) route_copy_kernel(const int32_t *__restrict__ anc_sys,
                                                         int32_t *__restrict__ anc, int32_t G,
                                                         const int32_t *__restrict__ seg_chunk,
                                                         const int64_t *__restrict__ seg_tick,
                                                         const int64_t *__restrict__ seg_dst,
                                                         const int64_t *__restrict__ seg_len, int64_t N,
                                                         DevSummary *__restrict__ sum)
{
    __shared__ int32_t sseg;
    const int32_t nb = sum->n_chunks;
    const int32_t nseg = seg_chunk[2 * G + 1];
    const int lane = threadIdx.x & 31;
    for (int32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        if (threadIdx.x < 32) {
            int32_t lo = 0, hi = nseg;  // seg_chunk[lo] <= b < seg_chunk[hi] (hi may be nseg)
            while (hi - lo > 1) {
                const int32_t step = (hi - lo + 31) / 32;
                const int32_t p = lo + lane * step;
                const bool le = p < hi && __ldg(seg_chunk + p) <= b;
                const unsigned m = __ballot_sync(0xffffffffu, le);  // a prefix of the lanes
                const int32_t last = 31 - __clz(m);
                lo = lo + last * step;
                const int32_t nh = lo + step;
                hi = nh < hi ? nh : hi;
            }
            if (lane == 0)
                sseg = lo;
        }
        __syncthreads();
        const int32_t s = sseg;
        const int64_t k0 = (int64_t)(b - __ldg(seg_chunk + s)) * COPY_CHUNK;
        const int64_t len = __ldg(seg_len + s);
        const int64_t k1 = (k0 + COPY_CHUNK < len) ? k0 + COPY_CHUNK : len;
        const int64_t src = __ldg(seg_tick + s), dst = __ldg(seg_dst + s);
        if (src < 0 || dst < 0 || k0 < 0 || src + k1 > N || dst + k1 > N) {
            if (threadIdx.x == 0)
                atomicOr(&sum->flags, FLAG_INTERNAL);  // inconsistent schedule: never write out of bounds
        } else {
            // four loads in flight per thread before the stores
            for (int64_t k = k0 + threadIdx.x; k < k1; k += 4 * (int64_t)blockDim.x) {
                int32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t kk = k + q * (int64_t)blockDim.x;
                    v[q] = kk < k1 ? __ldg(anc_sys + src + kk) : 0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t kk = k + q * (int64_t)blockDim.x;
                    if (kk < k1)
                        anc[dst + kk] = v[q];
                }
            }
        }
        __syncthreads();  // sseg is rewritten for the next item
    }
}

// ------------------------------------------------------------------- RNA
// One block per group: group max, fixed-point weights, local total and group
// weight (FP64 against the global total of the step), local systematic
// tickets, then every offspring is written to its slot -- the last `mig`
// slots of the group go to the tail of the next group of the ring (group
// g + 1 mod G, or succ[g] for ARNA's ring).
__global__ void __launch_bounds__(TILE_THREADS, 4) rna_kernel(
    const float *__restrict__ lw, int64_t N, int32_t G, const int64_t *__restrict__ goff,
    const int32_t *__restrict__ succ, DevSummary *sum, double ess_thr, uint64_t seed, uint32_t fid, uint32_t frame,
    int32_t *__restrict__ anc, float *__restrict__ lwp)
{
    if (kept_by_ess(sum, ess_thr))
        return;
    const int64_t mig = sum->mig;
    extern __shared__ uint64_t fill_smem[];  // FILL_SMEM_BYTES
    uint64_t *C = fill_smem;
    uint16_t *stage = reinterpret_cast<uint16_t *>(fill_smem + TILE_SMEM_U64);
    __shared__ uint64_t red[33];
    __shared__ float smf[8];
    __shared__ double lwg_s;
    __shared__ uint64_t Qs, us, qNs;
    __shared__ uint32_t qRs;
    __shared__ Divisor dvs;
    const int32_t g = blockIdx.x;
    const int64_t lo = goff[g], sz = goff[g + 1] - lo;
    if (sz <= 0)
        return;
    const int32_t gn = succ ? succ[g] : (g + 1) % G;
    const int64_t gn_lo = goff[gn], gn_sz = goff[gn + 1] - gn_lo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto dest = [&](int64_t s2) -> int64_t {
        return (s2 < sz - mig) ? lo + s2 : gn_lo + gn_sz - mig + (s2 - (sz - mig));
    };
    if (sz <= TILE) {
        // the whole group in one tile: its weights are loaded once and kept
        // in registers for the maximum, the sum of e^(lw - Mg), and the
        // quantised scan (whose total is the group's Q)
        const int n = (int)sz;
        float v[TILE_LOADS];
        tile_load(lw, lo, n, v);
        float m = -INFINITY;
#pragma unroll
        for (int k = 0; k < TILE_LOADS; ++k)
            m = fmaxf(m, v[k]);
        m = warp_max(m);
        if (lane == 0)
            smf[warp] = m;
        __syncthreads();
        float Mg = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            Mg = fmaxf(Mg, smf[w]);
        float es = 0.0f;
#pragma unroll
        for (int k = 0; k < TILE_LOADS; ++k)
            if (v[k] > -INFINITY)
                es += __expf(v[k] - Mg);
        es = warp_sum(es);
        __syncthreads();  // every thread has read smf
        if (lane == 0)
            smf[warp] = es;
        const int s = scale_bits(sz);
        uint64_t q[TILE_ITEMS];
        tile_quantise(v, Mg, s, C, q);  // its barriers also publish smf
        const uint64_t Qg = tile_scan(q, C, red);
        if (threadIdx.x == 0) {
            float e = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                e += smf[w];
            dvs = make_divisor((uint32_t)sz);
            qNs = Qg / (uint64_t)sz;
            qRs = (uint32_t)(Qg % (uint64_t)sz);
            if (Qg == 0ull) {
                lwg_s = -INFINITY;
                us = 0ull;
            } else {
                lwg_s = ((double)Mg + log((double)e)) - sum->log_total - log((double)sz);
                us = ticket_offset(seed, fid, frame, PURPOSE_GROUP, (uint32_t)g, Qg);
            }
        }
        __syncthreads();
        const float lwg = (float)lwg_s;
        if (Qg == 0ull) {  // no usable weight in the group: it keeps its slots
            for (int64_t s2 = threadIdx.x; s2 < sz; s2 += blockDim.x) {
                const int64_t d = dest(s2);
                if (!PPF_DCHECK(d >= 0 && d < N, &sum->flags, FLAG_INTERNAL))
                    continue;
                anc[d] = (int32_t)(lo + s2);
                lwp[d] = lwg;
            }
            return;
        }
        const TicketGrid tg = ticket_grid(Qg, us, qNs, qRs, dvs);
        ticket_parents_staged(C, n, 0, tg, 0, sz, stage, [&](int64_t j, int i) {
            const int64_t d = dest(j);
            if (!PPF_DCHECK(d >= 0 && d < N && i >= 0 && i < n, &sum->flags, FLAG_INTERNAL))
                return;
            anc[d] = (int32_t)(lo + i);
            lwp[d] = lwg;
        });
        return;
    }
    // pass 1: group maximum
    float m = -INFINITY;
    for (int64_t i = threadIdx.x; i < sz; i += blockDim.x)
        m = fmaxf(m, __ldg(lw + lo + i));
    m = warp_max(m);
    if (lane == 0)
        smf[warp] = m;
    __syncthreads();
    float Mg = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        Mg = fmaxf(Mg, smf[w]);
    __syncthreads();
    const int s = scale_bits(sz);
    // pass 2: total fixed-point weight and sum of e^(lw - Mg)
    uint64_t qs = 0;
    float es = 0.0f;
    for (int64_t i = threadIdx.x; i < sz; i += 2 * (int64_t)blockDim.x) {
        // two strided elements at a time (the sum of e^(lw - Mg) keeps its order)
        const int64_t i2 = i + blockDim.x;
        const float v = __ldg(lw + lo + i);
        const float w = (i2 < sz) ? __ldg(lw + lo + i2) : -INFINITY;
        uint64_t a, b;
        quantise2(v, w, Mg, s, a, b);
        qs += a + b;
        if (v > -INFINITY)
            es += __expf(v - Mg);
        if (w > -INFINITY)
            es += __expf(w - Mg);
    }
    uint64_t Qg;
    block_excl_scan_u64(qs, red, &Qg);
    es = warp_sum(es);
    if (lane == 0)
        smf[warp] = es;
    __syncthreads();
    if (threadIdx.x == 0) {
        float e = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            e += smf[w];
        Qs = Qg;
        dvs = make_divisor((uint32_t)sz);
        qNs = Qg / (uint64_t)sz;
        qRs = (uint32_t)(Qg % (uint64_t)sz);
        if (Qg == 0ull) {
            lwg_s = -INFINITY;
            us = 0ull;
        } else {
            lwg_s = ((double)Mg + log((double)e)) - sum->log_total - log((double)sz);
            us = ticket_offset(seed, fid, frame, PURPOSE_GROUP, (uint32_t)g, Qg);
        }
    }
    __syncthreads();
    const uint64_t Q = Qs, u = us;
    const float lwg = (float)lwg_s;
    if (Q == 0ull) {  // no usable weight in the group: it keeps its slots
        for (int64_t s2 = threadIdx.x; s2 < sz; s2 += blockDim.x) {
            const int64_t d = dest(s2);
            if (!PPF_DCHECK(d >= 0 && d < N, &sum->flags, FLAG_INTERNAL))
                continue;
            anc[d] = (int32_t)(lo + s2);
            lwp[d] = lwg;
        }
        return;
    }
    const TicketGrid tg = ticket_grid(Q, u, qNs, qRs, dvs);
    // pass 3: chunks of TILE particles; the tickets of chunk [c0, c0 + n) are
    // [T(carry), T(carry + total)) with T the local ticket count of n = sz.
    uint64_t carry = 0;
    for (int64_t c0 = 0; c0 < sz; c0 += TILE) {
        const int n = (int)(sz - c0 < TILE ? sz - c0 : TILE);
        uint64_t q[TILE_ITEMS];
        tile_weights(lw, lo + c0, n, Mg, s, C, q);
        const uint64_t tot = tile_scan(q, C, red);
        const int64_t t_lo = tickets_below(carry, sz, u, Q);
        const int64_t t_hi = tickets_below(carry + tot, sz, u, Q);
        ticket_parents_staged(C, n, carry, tg, t_lo, t_hi, stage, [&](int64_t j, int i) {
            const int64_t d = dest(j);
            if (!PPF_DCHECK(d >= 0 && d < N && i >= 0 && i < n, &sum->flags, FLAG_INTERNAL))
                return;
            anc[d] = (int32_t)(lo + c0 + i);
            lwp[d] = lwg;
        });
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) rna_prep_kernel(const int64_t *__restrict__ goff, int32_t G, float alpha,
                                                        DevSummary *sum, double ess_thr)
{
    __shared__ long long smx[32], smn[32];
    long long mx = 0, mn = INT64_MAX;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        const long long sz = goff[g + 1] - goff[g];
        mx = sz > mx ? sz : mx;
        mn = sz < mn ? sz : mn;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long a = __shfl_xor_sync(0xffffffffu, mx, o);
        const long long b = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = a > mx ? a : mx;
        mn = b < mn ? b : mn;
    }
    if ((threadIdx.x & 31) == 0) {
        smx[threadIdx.x >> 5] = mx;
        smn[threadIdx.x >> 5] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = INT64_MAX;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = smx[w] > a ? smx[w] : a;
            b = smn[w] < b ? smn[w] : b;
        }
        const bool kept = kept_by_ess(sum, ess_thr);  // N_eff test: no resampling, no exchange
        const int64_t mig = kept ? 0 : (int64_t)floor((double)alpha * (double)b);
        sum->mig = mig;
        sum->max_group = a;
        sum->min_group = b;
        sum->links = (G > 1 && mig > 0) ? G : 0;
        sum->moved = (G > 1) ? mig * G : 0;
        sum->degenerate = kept ? 1 : 0;
        if (kept)
            sum->flags |= FLAG_KEPT;
    }
}

// ------------------------------------------------------------------ ARNA
// One block, after the RPA tile passes have counted the tickets below every
// group start (Tg): the involved groups (proportional allocation gives them
// at least their own size), the adaptive number of migrants
// mig = floor(alpha (G - |I|) min_g n_g / G) (FP64, in that order), and the
// ring -- redrawn when the step's log-evidence is negative (the object
// counts as lost): the groups in increasing order of the first Philox word of
// (seed; g, frame, filter, RING), ties by index (the merge sort of
// word << 32 | g).  Then every group's successor on the ring.
// Dynamic shared memory: sort_smem_bytes(G) (G <= MAX_SCHED_GROUPS).
__global__ void __launch_bounds__(1024) arna_prep_kernel(const int64_t *__restrict__ goff, int32_t G, float alpha,
                                                         DevSummary *sum, double ess_thr,
                                                         const int64_t *__restrict__ Tg, int32_t *__restrict__ ring,
                                                         int32_t *__restrict__ succ, uint64_t seed, uint32_t fid,
                                                         uint32_t frame)
{
    extern __shared__ uint64_t sm[];
    __shared__ long long smx[32], smn[32];
    __shared__ int sinv[32];
    __shared__ bool s_lost;
    const bool kept = kept_by_ess(sum, ess_thr);  // N_eff test: no resampling, no exchange, ring kept
    const bool usable = !kept && sum->Q != 0ull;  // Tg holds the tickets only when some weight is usable
    long long mx = 0, mn = INT64_MAX;
    int inv = 0;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        const long long sz = goff[g + 1] - goff[g];
        mx = sz > mx ? sz : mx;
        mn = sz < mn ? sz : mn;
        if (usable && Tg[g + 1] - Tg[g] >= sz)
            ++inv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const long long a = __shfl_xor_sync(0xffffffffu, mx, o);
        const long long b = __shfl_xor_sync(0xffffffffu, mn, o);
        mx = a > mx ? a : mx;
        mn = b < mn ? b : mn;
        inv += __shfl_xor_sync(0xffffffffu, inv, o);
    }
    if ((threadIdx.x & 31) == 0) {
        smx[threadIdx.x >> 5] = mx;
        smn[threadIdx.x >> 5] = mn;
        sinv[threadIdx.x >> 5] = inv;
    }
    if (threadIdx.x == 0)
        s_lost = !kept && !(sum->log_evidence >= 0.0);
    __syncthreads();
    if (s_lost) {
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            const uint4 r = draw(seed, (uint32_t)g, frame, fid, PURPOSE_RING, 0);
            sm[g] = ((uint64_t)r.x << 32) | (uint32_t)g;
        }
        __syncthreads();
        block_sort_u64(sm, G, sm, G);
        for (int p = threadIdx.x; p < G; p += blockDim.x)
            ring[p] = (int32_t)(uint32_t)sm[p];
        __syncthreads();
    }
    for (int p = threadIdx.x; p < G; p += blockDim.x)
        succ[ring[p]] = ring[(p + 1) % G];
    if (threadIdx.x == 0) {
        long long a = 0, b = INT64_MAX;
        int in = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = smx[w] > a ? smx[w] : a;
            b = smn[w] < b ? smn[w] : b;
            in += sinv[w];
        }
        const int64_t mig =
            kept ? 0 : (int64_t)floor((double)alpha * (double)(G - in) * (double)b / (double)G);
        sum->mig = mig;
        sum->involved = in;
        sum->max_group = a;
        sum->min_group = b;
        sum->links = (G > 1 && mig > 0) ? G : 0;
        sum->moved = (G > 1) ? mig * G : 0;
        sum->degenerate = kept ? 1 : 0;
        if (kept)
            sum->flags |= FLAG_KEPT;
        if (s_lost)
            sum->flags |= FLAG_RING;
    }
}

// ancestors / starting log-weights the next step will use
__global__ void pending_kernel(int64_t N, int mode, const int32_t *__restrict__ anc, const float *__restrict__ lwp,
                               const float *__restrict__ lw_cur, const int32_t *__restrict__ degenerate,
                               int32_t *__restrict__ anc_out, float *__restrict__ lwp_out)
{
    const int m = (mode != MODE_CARRY && *degenerate) ? MODE_CARRY : mode;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        if (anc_out)
            anc_out[i] = (m == MODE_CARRY) ? (int32_t)i : anc[i];
        if (lwp_out)
            lwp_out[i] = (m == MODE_CARRY) ? lw_cur[i] : (m == MODE_UNIFORM ? 0.0f : lwp[i]);
    }
}

__global__ void identity_kernel(int32_t *__restrict__ a, int64_t N)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

__global__ void fill_f32_kernel(float *__restrict__ a, int64_t N, float v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

// ---------------------------------------------------------------- launchers
// Opt the dynamic-shared-memory kernels of this file into their sizes (current
// device; called when a context is created).
cudaError_t resample_kernel_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)FILL_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fill_tiles_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FILL_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fill_tiles_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FILL_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rna_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FILL_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(group_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FILL_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(schedule_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SORT_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(arna_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SORT_SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tile_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(uint64_t) * (SCAN_SMEM_TILES + 1)));
    return e;
}

// The tile prefix and the draw (one block), then the tickets below every
// tile and group start and the fill's list of further runs (one thread each).
// rpa: 0 systematic, 1 RPA, 2 ARNA.
static void launch_tile_tickets(ppf_ctx *c, double ess_thr, int rpa)
{
    const int T = c->T;
    const int32_t st_tiles = T <= SCAN_SMEM_TILES ? T : 0;
    const Divisor nd = make_divisor((uint32_t)c->N);
    int2 *extra = reinterpret_cast<int2 *>(c->sc.extra);
    // up to a tile or a group per thread, the block counts the tickets itself
    // (one launch less); beyond, one thread per tile and group does
    const bool one_block = T <= 1024 && (!rpa || c->G <= 1024);
    tile_scan_kernel<<<1, 1024, sizeof(uint64_t) * (st_tiles + 1), c->stream>>>(
        c->N, T, c->sc.Qt, c->sc.Ct, c->sc.Tt, c->sc.item_off, nullptr, c->sum, ess_thr, c->m.seed, c->m.filter_id,
        (uint32_t)c->last_frame, c->goff, c->G, rpa, c->sc.Cbl, c->sc.Tg, st_tiles, nd, one_block ? 0 : 1, extra);
    if (one_block)
        return;
    const int n = (rpa && c->G > T ? c->G : T) + 1;
    tile_tickets_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(c->N, T, c->sc.Ct, c->sc.Tt, c->sum, nd, c->goff,
                                                                c->G, rpa, c->sc.Cbl, c->sc.Tg, extra);
    c->launches += 1;
}

// The RPA schedule on the context's side stream, after the tile scan (an
// event on the main stream), its completion recorded in ev_sched.
static cudaError_t launch_schedule(ppf_ctx *c, int scheme, bool two_stage)
{
    cudaError_t e = cudaEventRecord(c->ev_scan, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(c->side_stream, c->ev_scan, 0);
    if (e != cudaSuccess)
        return e;
    SchedArgs A;
    A.N = c->N;
    A.G = c->G;
    A.scheme = two_stage ? scheme - (PPF_RPA2_GS - PPF_RPA_GS) : scheme;  // the schedule
    A.goff = c->goff;
    A.goff_new = c->goff_new;
    A.Tg = c->sc.Tg;
    A.key = c->sc.skey;
    A.val = c->sc.sval;
    A.seg_chunk = c->sc.seg_chunk;
    A.seg_tick = c->sc.seg_tick;
    A.seg_dst = c->sc.seg_dst;
    A.seg_len = c->sc.seg_len;
    A.sum = c->sum;
    A.links_only = A.scheme != PPF_RPA_LGS;
    A.bl = balanced_layout(c->N, c->G);
    const size_t sched_smem = sched_smem_bytes(c->G);
    schedule_kernel<<<1, 1024, sched_smem, c->side_stream>>>(A);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaEventRecord(c->ev_sched, c->side_stream);
    return e;
}

cudaError_t launch_resample_global(ppf_ctx *c, int scheme, double ess_thr)
{
    const bool rpa = (scheme != PPF_SYSTEMATIC);
    const float *lw = c->state[c->cur] + 5 * c->N;
    const int T = c->T;
    prof_mark(c, PH_RESAMPLE, 0);
    c->launches += rpa ? 5 : 3;
    if (rpa)
        tile_group_totals_kernel<<<T, TILE_THREADS, 0, c->stream>>>(lw, c->N, c->sum, ess_thr, c->sc.Qt, c->goff,
                                                                    c->G, c->sc.Cbl, c->sc.tile_g);
    else  // five blocks per SM (47 registers), each tile's loads one tile ahead
        tile_totals_kernel<<<T < 5 * c->num_sms ? T : 5 * c->num_sms, TILE_THREADS, 0, c->stream>>>(
            lw, c->N, c->sum, ess_thr, c->sc.Qt);
    launch_tile_tickets(c, ess_thr, rpa ? 1 : 0);
    int32_t *out = rpa ? c->anc_sys : c->anc;
    const bool two_stage = (scheme >= PPF_RPA2_GS && scheme <= PPF_RPA2_LGS);
    if (rpa) {
        // The routing schedule needs only the tile scan (offspring counts per
        // group), not the fill: it runs on a side stream, one block on one
        // SM, while the fill runs on the others; the copy joins them.
        cudaError_t e0 = launch_schedule(c, scheme, two_stage);
        if (e0 != cudaSuccess)
            return e0;
    }
    // GS and SGS: the kept tickets go straight to their balanced slots
    const bool kept_direct = rpa && scheme != PPF_RPA_LGS && scheme != PPF_RPA2_LGS;
    if (two_stage) {  // stage 2: every group draws its own offspring
        int4 *split = reinterpret_cast<int4 *>(c->sc.split);
        group_grid_kernel<<<(c->G + 255) / 256, 256, 0, c->stream>>>(
            c->N, c->G, c->goff, c->sc.Tg, c->sc.Ct, c->sc.Cbl, c->sum, ess_thr, c->m.seed, c->m.filter_id,
            (uint32_t)c->last_frame, c->sc.ggrid, split, balanced_layout(c->N, c->G));
        split_runs_kernel<<<c->num_sms, 256, 0, c->stream>>>(c->sc.Ct, c->sc.ggrid, split, c->sum, ess_thr);
        const int n_workers = 4 * c->num_sms;
        group_fill_kernel<<<n_workers + c->G, TILE_THREADS, FILL_SMEM_BYTES, c->stream>>>(
            lw, c->N, c->G, c->sc.Tg, c->sc.Ct, c->sc.ggrid, split, n_workers, c->sum, ess_thr, out,
            kept_direct ? c->anc : nullptr, balanced_layout(c->N, c->G), scale_bits(c->N));
        c->launches += 2;
    } else {
        // block t < T: tile t's first run of tickets; the rest: the listed further runs
        const int max_items = T + (int)(c->N / ITEM_TICKETS) + 1;
        const int2 *extra = reinterpret_cast<const int2 *>(c->sc.extra);
        if (kept_direct) {
            const KeptRoute kr{c->anc, c->sc.Tg, c->sc.tile_g, c->G, balanced_layout(c->N, c->G)};
            fill_tiles_kernel<true><<<max_items, TILE_THREADS, FILL_SMEM_BYTES, c->stream>>>(
                lw, c->N, T, make_divisor((uint32_t)c->N), c->sum, c->sc.Ct, c->sc.Tt, extra, out, kr);
        } else {
            const KeptRoute none{nullptr, nullptr, nullptr, 0, Balanced{0, 0}};
            fill_tiles_kernel<false><<<max_items, TILE_THREADS, FILL_SMEM_BYTES, c->stream>>>(
                lw, c->N, T, make_divisor((uint32_t)c->N), c->sum, c->sc.Ct, c->sc.Tt, extra, out, none);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !rpa) {
        prof_mark(c, PH_RESAMPLE, 1);
        return e;
    }
    e = cudaStreamWaitEvent(c->stream, c->ev_sched, 0);  // join the schedule
    if (e != cudaSuccess)
        return e;
    const int max_chunks = 2 * c->G + 1 + (int)((c->N + COPY_CHUNK - 1) / COPY_CHUNK);
    const int gcopy = max_chunks < 8 * c->num_sms ? max_chunks : 8 * c->num_sms;
    route_copy_kernel<<<gcopy, 256, 0, c->stream>>>(c->anc_sys, c->anc, c->G, c->sc.seg_chunk,
                                                         c->sc.seg_tick, c->sc.seg_dst, c->sc.seg_len, c->N,
                                                         c->sum);
    prof_mark(c, PH_RESAMPLE, 1);
    return cudaGetLastError();
}

cudaError_t launch_resample_rna(ppf_ctx *c, float alpha, double ess_thr)
{
    const float *lw = c->state[c->cur] + 5 * c->N;
    prof_mark(c, PH_RESAMPLE, 0);
    rna_prep_kernel<<<1, 1024, 0, c->stream>>>(c->goff, c->G, alpha, c->sum, ess_thr);
    rna_kernel<<<c->G, TILE_THREADS, FILL_SMEM_BYTES, c->stream>>>(lw, c->N, c->G, c->goff, nullptr, c->sum, ess_thr,
                                                                   c->m.seed, c->m.filter_id,
                                                                   (uint32_t)c->last_frame, c->anc, c->lwp);
    prof_mark(c, PH_RESAMPLE, 1);
    c->launches += 2;
    return cudaGetLastError();
}

// ARNA: the RPA tile passes count each group's proportional offspring, one
// block settles the exchange and the ring, then RNA's per-group kernel.
cudaError_t launch_resample_arna(ppf_ctx *c, float alpha, double ess_thr)
{
    const float *lw = c->state[c->cur] + 5 * c->N;
    const int T = c->T;
    prof_mark(c, PH_RESAMPLE, 0);
    tile_group_totals_kernel<<<T, TILE_THREADS, 0, c->stream>>>(lw, c->N, c->sum, ess_thr, c->sc.Qt, c->goff, c->G,
                                                                c->sc.Cbl, c->sc.tile_g);
    launch_tile_tickets(c, ess_thr, 2);
    arna_prep_kernel<<<1, 1024, sort_smem_bytes(c->G), c->stream>>>(
        c->goff, c->G, alpha, c->sum, ess_thr, c->sc.Tg, c->ring, c->succ, c->m.seed, c->m.filter_id,
        (uint32_t)c->last_frame);
    rna_kernel<<<c->G, TILE_THREADS, FILL_SMEM_BYTES, c->stream>>>(lw, c->N, c->G, c->goff, c->succ, c->sum, ess_thr,
                                                                   c->m.seed, c->m.filter_id,
                                                                   (uint32_t)c->last_frame, c->anc, c->lwp);
    prof_mark(c, PH_RESAMPLE, 1);
    c->launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_pending(ppf_ctx *c, int32_t *anc_out, float *lwp_out)
{
    const int grid = (int)((c->N + 255) / 256 < 8192 ? (c->N + 255) / 256 : 8192);
    c->launches += 1;
    pending_kernel<<<grid, 256, 0, c->stream>>>(c->N, c->mode, c->anc, c->lwp, c->state[c->cur] + 5 * c->N,
                                                &c->sum->degenerate, anc_out, lwp_out);
    return cudaGetLastError();
}

cudaError_t launch_identity(ppf_ctx *c, int32_t *dst)
{
    const int grid = (int)((c->N + 255) / 256 < 8192 ? (c->N + 255) / 256 : 8192);
    c->launches += 1;
    identity_kernel<<<grid, 256, 0, c->stream>>>(dst, c->N);
    return cudaGetLastError();
}

// the ppf_estimate_t fields of the device summary (for ppf_estimate_async)
__global__ void format_estimate_kernel(const DevSummary *__restrict__ sum, ppf_estimate_t *__restrict__ out)
{
    ppf_estimate_t e;
    for (int i = 0; i < 5; ++i)
        e.mean[i] = sum->mean[i];
    e.log_evidence = sum->log_evidence;
    e.ess = sum->ess;
    e.max_log_weight = sum->max_lw;
    e.frame = sum->frame;
    e.status_flags = sum->flags;
    e.links = sum->links;
    e.moved = sum->moved;
    e.max_group = sum->max_group;
    e.min_group = sum->min_group;
    *out = e;
}

cudaError_t launch_format_estimate(ppf_ctx *c)
{
    format_estimate_kernel<<<1, 1, 0, c->stream>>>(c->sum, c->est_dev);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_fill_f32(ppf_ctx *c, float *dst, float v)
{
    const int grid = (int)((c->N + 255) / 256 < 8192 ? (c->N + 255) / 256 : 8192);
    fill_f32_kernel<<<grid, 256, 0, c->stream>>>(dst, c->N, v);
    return cudaGetLastError();
}

}  // namespace ppf
