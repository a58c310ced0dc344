// update.cu — RobustPrune, Publish-based update kernels: forward edges and
// own slab (Algorithm 2), reverse-edge offers, the refine pass, tombstoning
// and repair (Algorithm 3), compaction and reclaim (Algorithm 4).
//
// Deterministic mode groups offers by target (a stable radix sort by target
// id keeps sources ascending) and lets one warp fold a target's offers in
// order and publish once.  Lock-free mode gives each offer its own warp,
// which snapshots the target, builds the new list and publishes it with a
// compare-and-swap, retrying up to the attempt budget (Algorithm 1).
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace etale {

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// ---------------------------------------------------------------------------
// Row staging: the rows of the first `ns` candidates are copied into shared
// memory by bulk (TMA) copies completing on the warp's mbarrier; later
// candidates are read from global memory.
// ---------------------------------------------------------------------------
struct Stage {
    float *rows;     // ns_cap x mp floats, 16-byte aligned (nullptr: no staging)
    int ns_cap;
    u64 *bar;        // this warp's mbarrier
    u32 phase;
    bool timeout;
    char *gram;      // gram_bytes(gram_rows, mp) for the tensor-core Gram path (nullptr: canonical path)
    int gram_rows;   // candidates the Gram buffer holds (a multiple of 16, <= GRAM_NL)
    u64 wk_rows, wk_state;   // this warp's work tallies (see WK_*), added by stage_done
};

// Tensor-core Gram tile: up to 64 candidates, K staged 128 columns at a time
// as bf16 rows of 256 bytes with no pad; the 16-byte chunk c of row r sits at
// chunk c ^ (r & 7), so the eight rows an ldmatrix phase reads at one column
// fall in eight distinct bank groups.  The 64 x 64 fp32 result (row stride
// GRAM_N floats, also 256 bytes) reuses the same bytes.
constexpr int GRAM_N = 64;
constexpr int GRAM_RB = 256;   // bytes per staged row (128 bf16 columns)
// The large path (more than GRAM_N rows) keeps rows of GRAM_RS_LG bf16 (a
// 16-byte pad: conflict-free ldmatrix without a swizzle), so that a whole
// row block lands with one bulk copy per row.
constexpr int GRAM_RS_LG = 136;
__host__ __device__ inline size_t gram_rowb(u32 rows) { return rows > (u32)GRAM_N ? (size_t)GRAM_RS_LG * 2 : GRAM_RB; }
__host__ __device__ inline u32 gram_xoff(int r, int chunk) { return (u32)(r * GRAM_RB + ((chunk ^ (r & 7)) << 4)); }
// Byte offset, in a Gram buffer for `rows` candidates, of the partial sums
// that rows longer than one 128-column block keep between blocks: after the
// bf16 rows (or the table over them), a (norm, rho) pair per candidate and
// the large path's domination masks.  rows is a multiple of 16.
__host__ __device__ inline size_t gram_part_off(u32 rows) {
    const size_t b = (size_t)rows * gram_rowb(rows) + (size_t)rows * 8;
    return rows > (u32)GRAM_N ? b + (size_t)rows * 16 : b;
}
// Shared-memory bytes of a Gram buffer for `rows` candidates of mp columns;
// 0 rows = no buffer.  With more than one column block, a small-path buffer
// (rows <= GRAM_N) also holds one accumulator fragment (32 lanes x 16 bytes)
// per upper-triangle tile: nm (nm + 1) tiles for nm = rows / 16 stripes.
__host__ __device__ inline size_t gram_bytes(u32 rows, u32 mp) {
    if (!rows) return 0;
    const size_t nm = rows / 16;
    return gram_part_off(rows) + (mp > 128 && rows <= (u32)GRAM_N ? nm * (nm + 1) * 512 : 0);
}
// First tile slot of stripe mt among the partial sums (stripe mt holds the
// tiles nt = 2 mt .. 2 nmr - 1, nmr = rows / 16).
__device__ __forceinline__ int gram_part_slot(int mt, int nmr) { return mt * (2 * nmr + 1 - mt); }
constexpr int GRAM_NL = 128;   // candidates of the large (mask) path
// The Gram variant (see warp_prune) of a kernel whose buffer holds gram_rows rows of mp columns.
inline int gram_variant(u32 gram_rows, u32 mp) { return gram_rows > (u32)GRAM_N ? 1 : (gram_rows && mp > 128 ? 2 : 0); }
// Gram rows for a kernel whose prunes see at most max_n candidates (0: the
// Gram path is off or cannot hold them).  Above GRAM_N rows the kernel runs
// the large path (warp_prune_masks).
inline u32 gram_rows_for(u32 on, u32 max_n) { return on && max_n <= (u32)GRAM_NL ? (max_n + 15) / 16 * 16 : 0; }
// Scratch that is dead whenever the Gram buffer is live (list compaction before
// a prune, the canonical prune's arrays, a prune's output, written after its
// last read of the buffer) lives inside the Gram buffer's row bytes if it fits.
__host__ __device__ inline bool gram_alias(u32 gram, size_t scratch) { return gram && scratch <= (size_t)gram * GRAM_RB; }

// Shared-memory bytes for a stage of ns rows plus its mbarrier.
__host__ __device__ inline size_t stage_bytes(u32 ns, u32 mp) { return al16((size_t)ns * mp * 4) + 16; }

// Carve a stage at p (16-byte aligned) and initialise the warp's mbarrier.
__device__ __forceinline__ Stage stage_init(char *p, u32 ns, u32 mp, char *gram = nullptr, u32 gram_rows = 0) {
    Stage st;
    st.rows = ns ? reinterpret_cast<float *>(p) : nullptr;
    st.ns_cap = (int)ns;
    st.bar = reinterpret_cast<u64 *>(p + al16((size_t)ns * mp * 4));
    st.phase = 0;
    st.timeout = false;
    st.gram = gram;
    st.gram_rows = (int)gram_rows;
    st.wk_rows = st.wk_state = 0;
    if (lane_id() == 0) mbar_init(st.bar, 1);
    __syncwarp();
    return st;
}

__device__ __forceinline__ void stage_done(const Dev &d, const Stage &st, int kind) {
    if (lane_id() != 0) return;
    if (st.timeout) atomicOr(&d.ctr[C_ERR], (u64)ERR_TIMEOUT);
    if (st.wk_rows) atomicAdd(&d.ctr[C_WK + 2 * kind], st.wk_rows);
    if (st.wk_state) atomicAdd(&d.ctr[C_WK + 2 * kind + 1], st.wk_state);
}

// Row bytes a prune of n candidates gathers: the bf16 copy on the Gram path
// when the index keeps one, else the fp32 rows.
__device__ __forceinline__ u64 prune_row_bytes(const Dev &d, const Stage &st, int n) {
    const bool b16 = st.gram && n <= st.gram_rows && d.xb;
    return (u64)n * (b16 ? 2ull * d.mb : 4ull * d.mp);
}

// Warps per block (<= 4) such that a block's shared memory stays <= 200 KB.
// Warps per block of the persistent update kernels: one.  Their shared memory
// is per warp (up to ~20 KB with the Gram tile), so one-warp blocks pack the
// SM by the warp instead of by four (11 warps instead of 8 at 19 KB).
inline int warps_for(size_t) { return 1; }

// Rows that fit a per-warp stage of `budget` bytes, capped at `want`.
inline u32 stage_cap(u32 mp, u32 want, u32 budget) {
    u32 cap = budget / (mp * 4u);
    return cap < want ? cap : want;
}

template <class IdOf>
__device__ __forceinline__ void stage_rows_by(const Dev &d, Stage &st, int ns, IdOf id_of) {
    const int lane = lane_id();
    if (ns <= 0) return;
    const u32 rowb = d.mp * 4;
    if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(st.bar, (u32)ns * rowb);
    }
    __syncwarp();
    for (int i = lane; i < ns; i += 32)
        bulk_g2s(st.rows + (size_t)i * d.mp, d.x + (size_t)id_of(i) * d.mp, rowb, st.bar);
    if (!mbar_wait(st.bar, st.phase, WAIT_LIMIT)) {
        st.timeout = true;
        mbar_wait(st.bar, st.phase, WAIT_LIMIT);
    }
    st.phase ^= 1u;
    __syncwarp();
}

__device__ __forceinline__ void stage_rows(const Dev &d, Stage &st, const u64 *ck, int ns) {
    stage_rows_by(d, st, ns, [&](int i) { return key_id(ck[i]); });
}


// ---------------------------------------------------------------------------
// Candidate Gram tile on the tensor cores (mma.sync m16n8k16, bf16 inputs,
// fp32 accumulation): G = X X^T for the n <= 64 candidate rows X, one warp.
// Squared L2 follows as (G_ii - G_ij) + (G_jj - G_ij), inner product as
// 1 - G_ij.  Inputs rounded to bf16 are exact for integer-valued data of
// magnitude <= 256, and so is every product and partial sum while the norms
// stay below 2^24; then each distance equals the canonical one bit for bit.
// ---------------------------------------------------------------------------

// ldmatrix row addresses in the swizzled tile: lane l reads (row, chunk
// 2 ks + (l >> 4)) with row & 7 = l & 7, so the chunk's byte offset in its row
// is (32 ks) ^ c0 with c0 = 16 ((l >> 4) ^ (l & 7)), shared by every row.
__device__ __forceinline__ u32 gram_c0(int lane) { return (u32)(((lane >> 4) ^ (lane & 7)) << 4); }

__device__ __forceinline__ void cp_async16(u32 dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage columns [128 kb, 128 kb + 128) of candidate rows [r_lo, r_hi) into the
// swizzled tile at xs, a lane per row and a 16-byte copy per chunk; chunks past
// the row's end are zeroed.  From the bf16 copy when there is one (the same
// round-to-nearest-even values), else converted from the fp32 rows.
__device__ __forceinline__ void gram_stage_rows(const Dev &d, const u64 *ck, int r_lo, int r_hi, int kb, u32 xs) {
    __syncwarp();   // earlier reads of these bytes are done
    const int lane = lane_id();
    const int cols = min(128, (int)d.mb - 128 * kb);   // d.mb is a multiple of 8
    const int nch = cols >> 3;
    for (int r = r_lo + lane; r < r_hi; r += 32) {
        const u32 id = key_id(ck[r]);
        if (d.xb) {
            const auto *src = d.xb + (size_t)id * d.mb + 128 * kb;
#pragma unroll 4
            for (int c = 0; c < 16; c++) {
                if (c < nch) cp_async16(xs + gram_xoff(r, c), src + 8 * c);
                else asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(xs + gram_xoff(r, c)), "r"(0u) : "memory");
            }
        } else {
            const float *src = d.x + (size_t)id * d.mp + 128 * kb;
            const int pc = min(128, (int)d.mp - 128 * kb) >> 2;   // float4 columns (d.mp is a multiple of 4)
#pragma unroll 1
            for (int c = 0; c < 16; c++) {
                float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
                if (2 * c < pc) v0 = *reinterpret_cast<const float4 *>(src + 8 * c);
                if (2 * c + 1 < pc) v1 = *reinterpret_cast<const float4 *>(src + 8 * c + 4);
                asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(xs + gram_xoff(r, c)),
                             "r"(pack_bf16(v0.x, v0.y)), "r"(pack_bf16(v0.z, v0.w)), "r"(pack_bf16(v1.x, v1.y)),
                             "r"(pack_bf16(v1.z, v1.w))
                             : "memory");
            }
        }
    }
    cp_async_wait_all();
    __syncwarp();
}

// Column swizzle of the Gram table: entry (r, c) sits at column c ^ gram_tsw(r),
// so the eight rows of an accumulator fragment store to four bank groups
// (two wavefronts instead of eight), while a walk along rows (lane h reading
// (h, h + 1 + k)) still hits 32 distinct banks.
__device__ __forceinline__ int gram_tsw(int r) { return (r & 3) << 3; }

// Writes the upper triangle (j >= i, in 16 x 8 tiles) of the n x n Gram into
// T (fp32, row stride GRAM_N, columns swizzled by gram_tsw) and the diagonal
// into nr2[i].x, with rho_i (the candidate's key distance) in nr2[i].y.
// Rows of one 128-column block (MB false) are staged once, then the stripes
// run in ascending order.  With several blocks (MB true) the blocks go
// outermost: each block of every row is staged once, and each stripe adds
// its products for the block to the buffer's partial sums (fp32; exact for
// the integer-valued data the tile is exact for).  T and the bf16 rows share
// `buf`: in the (last) block the stripes go in ascending order, and stripe
// mt's table rows (bytes [4096 mt, 4096 (mt + 1))) are the staged rows of
// that same stripe, which no later stripe reads (it reads rows >= 16 (mt + 1)).
// A stripe only needs the columns j >= 16 mt, because the prune reads
// T[head][j] for j > head.  Rows past n hold whatever the buffer held: an
// entry (i, j) reads rows i and j only, and no entry with i or j >= n is read.
template <bool MB>   // rows span more than one 128-column block
__device__ void warp_gram(const Dev &d, const u64 *ck, int n, char *buf, int rows, Stage &st, float *&T, float2 *&nr2) {
    // The single-block form keeps its own loop nest: written as the
    // multi-block one with one block, it costs the 128-d kernels 10 to 20
    // registers and with them resident warps.
    if constexpr (!MB) {
        (void)st;
        const int lane = lane_id();
        T = reinterpret_cast<float *>(buf);
        nr2 = reinterpret_cast<float2 *>(buf + (size_t)rows * GRAM_RB);
        const int nm = (n + 15) >> 4, nn = (n + 7) >> 3;
        const int nkb = ((int)d.mp + 127) >> 7;
        const u32 xs = smem_addr(buf), c0 = gram_c0(lane);
        for (int mt = 0; mt < nm; mt++) {
            float acc[8][4];
#pragma unroll
            for (int b = 0; b < 8; b++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[b][c] = 0.f;
            for (int kb = 0; kb < nkb; kb++) {
                // rows [16 mt, n) of this column block: all rows once when one
                // block covers the row, else this stripe's and later ones per block
                if (nkb > 1 || mt == 0) gram_stage_rows(d, ck, 16 * mt, n, kb, xs);
#pragma unroll
                for (int ks = 0; ks < 8; ks++) {
                    u32 a0, a1, a2, a3;
                    const u32 ko = (u32)(32 * ks) ^ c0;
                    const int ar = 16 * mt + (lane & 7) + 8 * ((lane >> 3) & 1);
                    ldsm_x4(a0, a1, a2, a3, xs + (u32)ar * GRAM_RB + ko);
#pragma unroll
                    for (int nt = 0; nt < 8; nt += 2) {
                        if (nt < 2 * mt || nt >= nn) continue;
                        // matrices: (nt, k 0-7), (nt + 1, k 0-7), (nt, k 8-15), (nt + 1, k 8-15)
                        u32 b0, b1, b2, b3;
                        const int br = 8 * nt + (lane & 7) + 8 * ((lane >> 3) & 1);
                        ldsm_x4(b0, b1, b2, b3, xs + (u32)br * GRAM_RB + ko);
                        mma_bf16_16816(acc[nt], a0, a1, a2, a3, b0, b2);
                        mma_bf16_16816(acc[nt + 1], a0, a1, a2, a3, b1, b3);
                    }
                }
            }
            __syncwarp();
            // this stripe's table rows, over this stripe's staged rows (rows r and
            // r + 8 share the column swizzle)
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                if (nt < 2 * mt || nt >= nn) continue;
                const int r = 16 * mt + (lane >> 2), c = (8 * nt + 2 * (lane & 3)) ^ gram_tsw(r);
                *reinterpret_cast<float2 *>(T + r * GRAM_N + c) = make_float2(acc[nt][0], acc[nt][1]);
                *reinterpret_cast<float2 *>(T + (r + 8) * GRAM_N + c) = make_float2(acc[nt][2], acc[nt][3]);
            }
            __syncwarp();
        }
        for (int i = lane; i < n; i += 32) nr2[i] = make_float2(T[i * GRAM_N + (i ^ gram_tsw(i))], key_rho(ck[i]));
        __syncwarp();
    } else {
        (void)st;
        const int lane = lane_id();
        T = reinterpret_cast<float *>(buf);
        nr2 = reinterpret_cast<float2 *>(buf + (size_t)rows * GRAM_RB);
        float4 *part = reinterpret_cast<float4 *>(buf + gram_part_off((u32)rows));
        const int nm = (n + 15) >> 4, nn = (n + 7) >> 3, nmr = rows >> 4;
        const int nkb = MB ? ((int)d.mp + 127) >> 7 : 1;
        const u32 xs = smem_addr(buf), c0 = gram_c0(lane);
        for (int kb = 0; kb < nkb; kb++) {
            gram_stage_rows(d, ck, 0, n, kb, xs);
            const bool last = kb == nkb - 1;
            for (int mt = 0; mt < nm; mt++) {
                const int slot = gram_part_slot(mt, nmr) - 2 * mt;
                float acc[8][4];
#pragma unroll
                for (int b = 0; b < 8; b++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[b][c] = 0.f;
#pragma unroll
                for (int ks = 0; ks < 8; ks++) {
                    u32 a0, a1, a2, a3;
                    const u32 ko = (u32)(32 * ks) ^ c0;
                    const int ar = 16 * mt + (lane & 7) + 8 * ((lane >> 3) & 1);
                    ldsm_x4(a0, a1, a2, a3, xs + (u32)ar * GRAM_RB + ko);
#pragma unroll
                    for (int nt = 0; nt < 8; nt += 2) {
                        if (nt < 2 * mt || nt >= nn) continue;
                        // matrices: (nt, k 0-7), (nt + 1, k 0-7), (nt, k 8-15), (nt + 1, k 8-15)
                        u32 b0, b1, b2, b3;
                        const int br = 8 * nt + (lane & 7) + 8 * ((lane >> 3) & 1);
                        ldsm_x4(b0, b1, b2, b3, xs + (u32)br * GRAM_RB + ko);
                        mma_bf16_16816(acc[nt], a0, a1, a2, a3, b0, b2);
                        mma_bf16_16816(acc[nt + 1], a0, a1, a2, a3, b1, b3);
                    }
                }
                if constexpr (MB) {
                    // this block's products join the earlier blocks' sums
#pragma unroll
                    for (int nt = 0; nt < 8; nt++) {
                        if (nt < 2 * mt || nt >= nn) continue;
                        float4 *pp = part + (size_t)(slot + nt) * 32 + lane;
                        if (kb > 0) {
                            const float4 v = *pp;
                            acc[nt][0] = __fadd_rn(v.x, acc[nt][0]);
                            acc[nt][1] = __fadd_rn(v.y, acc[nt][1]);
                            acc[nt][2] = __fadd_rn(v.z, acc[nt][2]);
                            acc[nt][3] = __fadd_rn(v.w, acc[nt][3]);
                        }
                        if (!last) *pp = make_float4(acc[nt][0], acc[nt][1], acc[nt][2], acc[nt][3]);
                    }
                    if (!last) continue;
                }
                __syncwarp();
                // this stripe's table rows, over this stripe's staged rows (rows r and
                // r + 8 share the column swizzle)
#pragma unroll
                for (int nt = 0; nt < 8; nt++) {
                    if (nt < 2 * mt || nt >= nn) continue;
                    const int r = 16 * mt + (lane >> 2), c = (8 * nt + 2 * (lane & 3)) ^ gram_tsw(r);
                    *reinterpret_cast<float2 *>(T + r * GRAM_N + c) = make_float2(acc[nt][0], acc[nt][1]);
                    *reinterpret_cast<float2 *>(T + (r + 8) * GRAM_N + c) = make_float2(acc[nt][2], acc[nt][3]);
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < n; i += 32) nr2[i] = make_float2(T[i * GRAM_N + (i ^ gram_tsw(i))], key_rho(ck[i]));
        __syncwarp();
    }
}

// RobustPrune on a Gram table: same rule and order as warp_prune.  First the
// domination masks: row i's mask holds the later candidates j > i that i would
// drop (alpha^2 * d(i, j) <= rho(j)).  Lane l builds the mask of row l and,
// when n - 2 - l >= 32, of row n - 2 - l, walking each row's columns upward
// (lane l reads column row + 1 + k in step k: distinct banks).  The masks go
// to the last 512 bytes of the buffer's row area (the table is read by then); the
// greedy pass is a warp-uniform walk over a 64-bit alive mask (take the first
// alive candidate, clear the ones it drops), and the kept candidates are
// written out afterwards, a lane per candidate.
template <bool MB>
__device__ int warp_prune_gram(const Dev &d, const u64 *ck, int n, unsigned char *alive, u32 *out_id,
                               float *out_rho, Stage &st) {
    (void)alive;
    const int lane = lane_id();
    float *T;
    float2 *nr2;
    warp_gram<MB>(d, ck, n, st.gram, st.gram_rows, st, T, nr2);
    const float alpha2 = d.alpha2;
    const bool l2 = d.metric == 0;
    // (n_h - g) + (n_j - g): every intermediate stays as small as the result
    auto hit = [&](float nh, float g, int j) {
        const float2 v = nr2[j];
        const float dd = l2 ? __fadd_rn(__fsub_rn(nh, g), __fsub_rn(v.x, g)) : __fsub_rn(1.0f, g);
        return __fmul_rn(alpha2, dd) <= v.y;
    };
    u64 dom_a = 0ull, dom_b = 0ull;
    const int ra = lane, rb = n - 2 - lane;
    if (ra < n - 1) {
        const float *Ta = T + ra * GRAM_N;
        const float na = nr2[ra].x;
        const int sw = gram_tsw(ra);
#pragma unroll 4
        for (int j = ra + 1; j < n; j++)
            if (hit(na, Ta[j ^ sw], j)) dom_a |= 1ull << j;
    }
    if (rb >= 32) {
        const float *Tb = T + rb * GRAM_N;
        const float nb = nr2[rb].x;
        const int sw = gram_tsw(rb);
#pragma unroll 4
        for (int j = rb + 1; j < n; j++)
            if (hit(nb, Tb[j ^ sw], j)) dom_b |= 1ull << j;
    }
    __syncwarp();   // the table is read: its last bytes take the masks
    u64 *dsm = reinterpret_cast<u64 *>(st.gram + (size_t)st.gram_rows * GRAM_RB - GRAM_N * 8);
    if (ra < n) dsm[ra] = dom_a;
    if (rb >= 32) dsm[rb] = dom_b;
    if (lane == 0 && n - 1 >= 32) dsm[n - 1] = 0ull;   // the last row drops nothing
    // equal adjacent keys collapse to one
    u64 live = 0ull;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const u32 b = __ballot_sync(FULL, i < n && (i == 0 || ck[i] != ck[i - 1]));
        live |= (u64)b << i0;
    }
    __syncwarp();
    u64 kept = 0ull;
    int nout = 0;
    const int R = (int)d.R;
    while (nout < R && live) {
        const u64 low = live & (0ull - live);
        const int head = __ffsll((long long)live) - 1;
        kept |= low;
        nout++;
        live = (live ^ low) & ~dsm[head];
    }
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        if (i < n && (kept >> i & 1)) {
            const int pos = __popcll(kept & ((1ull << i) - 1));
            const u64 hk = ck[i];
            out_id[pos] = key_id(hk);
            out_rho[pos] = key_rho(hk);
        }
    }
    __syncwarp();
    return nout;
}
// RobustPrune on the tensor-core Gram for up to GRAM_NL candidates, with no
// table in shared memory: the Gram is built in 16-row stripes, last stripe
// first, so that by the time a stripe is converted the norms of every column
// it reads are known (this stripe's diagonal, or a later stripe's).  Each
// accumulator entry (i, j), j > i, becomes bit j of row i's domination mask
// (alpha^2 * d(i, j) <= rho(j)); the four lanes of a quad hold the columns of
// a row and OR their bits.  The greedy pass is the register walk of
// warp_prune_gram over 128-bit masks.  Same distances as warp_prune_gram:
// squared L2 as (G_ii - G_ij) + (G_jj - G_ij), inner product as 1 - G_ij.
template <int NT>   // tiles of 8 columns: 8 (n <= 64) or 16 (n <= 128)
__device__ int warp_prune_masks(const Dev &d, const u64 *ck, int n, u32 *out_id, float *out_rho, Stage &st) {
    const int lane = lane_id();
    const int rows = st.gram_rows;
    __nv_bfloat16 *X = reinterpret_cast<__nv_bfloat16 *>(st.gram);
    char *tail = st.gram + (size_t)rows * GRAM_RS_LG * 2;
    float2 *nr2 = reinterpret_cast<float2 *>(tail);   // .x: the norms (.y unused here)
    u64 *dom = reinterpret_cast<u64 *>(tail + (size_t)rows * 8);
    const int nm = (n + 15) >> 4, nn = (n + 7) >> 3;
    const int nkb = ((int)d.mp + 127) >> 7;
    const u32 xs = smem_addr(X);
    for (int mt = nm - 1; mt >= 0; mt--) {
        float acc[NT][4];
#pragma unroll
        for (int b = 0; b < NT; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[b][c] = 0.f;
        for (int kb = 0; kb < nkb; kb++) {
            if (nkb > 1 || mt == nm - 1) {
                // rows [r_lo, n) of columns [128 kb, 128 kb + 128): all rows once
                // when one block covers the row, else those of this stripe on
                const int r_lo = nkb > 1 ? 16 * mt : 0;
                __syncwarp();
                if (d.xb) {
                    const int cols = min(128, (int)d.mb - 128 * kb);
                    if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (cols < 128)
                        for (int z = lane; z < (n - r_lo) * 64; z += 32) {
                            const int r = r_lo + (z >> 6), c = (z & 63) * 2;
                            if (c >= cols) *reinterpret_cast<u32 *>(X + (size_t)r * GRAM_RS_LG + c) = 0u;
                        }
                    const int nr = n - r_lo;
                    if (lane == 0 && nr > 0) mbar_expect_tx(st.bar, (u32)(nr * cols * 2));
                    __syncwarp();
                    for (int r = r_lo + lane; r < n; r += 32)
                        bulk_g2s(X + (size_t)r * GRAM_RS_LG, d.xb + (size_t)key_id(ck[r]) * d.mb + 128 * kb,
                                 (u32)cols * 2, st.bar);
                    if (nr > 0) {
                        if (!mbar_wait(st.bar, st.phase, WAIT_LIMIT)) {
                            st.timeout = true;
                            mbar_wait(st.bar, st.phase, WAIT_LIMIT);   // let copies in flight land
                        }
                        st.phase ^= 1u;
                    }
                } else {
                    const int col = 128 * kb + 4 * lane;
                    for (int r = r_lo; r < n; r++) {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (col < (int)d.mp)
                            v = *reinterpret_cast<const float4 *>(d.x + (size_t)key_id(ck[r]) * d.mp + col);
                        *reinterpret_cast<uint2 *>(X + (size_t)r * GRAM_RS_LG + 4 * lane) =
                            make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int ks = 0; ks < 8; ks++) {
                u32 a0, a1, a2, a3;
                const int ar = 16 * mt + (lane & 7) + 8 * ((lane >> 3) & 1);
                const int ac = 16 * ks + 8 * (lane >> 4);
                ldsm_x4(a0, a1, a2, a3, xs + (u32)((ar * GRAM_RS_LG + ac) * 2));
#pragma unroll
                for (int nt = 0; nt < NT; nt += 2) {
                    if (nt < 2 * mt || nt >= nn) continue;
                    u32 b0, b1, b2, b3;
                    const int br = 8 * nt + (lane & 7) + 8 * (lane >> 4);
                    const int bc = 16 * ks + 8 * ((lane >> 3) & 1);
                    ldsm_x4(b0, b1, b2, b3, xs + (u32)((br * GRAM_RS_LG + bc) * 2));
                    mma_bf16_16816(acc[nt], a0, a1, a2, a3, b0, b1);
                    mma_bf16_16816(acc[nt + 1], a0, a1, a2, a3, b2, b3);
                }
            }
        }
        // this stripe's diagonal: entry (r, r) sits in tile 2 mt (rows r0) or 2 mt + 1 (rows r0 + 8)
        const int r0 = 16 * mt + (lane >> 2), r1 = r0 + 8, cq = 2 * (lane & 3);
        {
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int nt = 0; nt < NT; nt++) {
                if (nt == 2 * mt) d0 = cq == (lane >> 2) ? acc[nt][0] : acc[nt][1];
                if (nt == 2 * mt + 1) d1 = cq == (lane >> 2) ? acc[nt][2] : acc[nt][3];
            }
            const bool own = cq == (lane >> 2) || cq + 1 == (lane >> 2);
            if (own && r0 < n) nr2[r0].x = d0;
            if (own && r1 < n) nr2[r1].x = d1;
        }
        __syncwarp();
        const float n0 = r0 < n ? nr2[r0].x : 0.f, n1 = r1 < n ? nr2[r1].x : 0.f;
        u64 m0l = 0, m0h = 0, m1l = 0, m1h = 0;
#pragma unroll
        for (int nt = 0; nt < NT; nt++) {
            const bool tile = nt >= 2 * mt && nt < nn;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int r = e < 2 ? r0 : r1, c = 8 * nt + cq + (e & 1);
                const bool ok = tile && c > r && c < n;   // c < n implies r < n
                const int cc = ok ? c : 0;
                const float g = acc[nt][e];
                const float nr_ = e < 2 ? n0 : n1;
                const float dd = d.metric == 0 ? __fadd_rn(__fsub_rn(nr_, g), __fsub_rn(nr2[cc].x, g)) : __fsub_rn(1.0f, g);
                const bool hit = ok && __fmul_rn(d.alpha2, dd) <= key_rho(ck[cc]);
                const u64 bit = hit ? 1ull << (c & 63) : 0ull;
                if (e < 2) { if (8 * nt < 64) m0l |= bit; else m0h |= bit; }
                else { if (8 * nt < 64) m1l |= bit; else m1h |= bit; }
            }
        }
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            m0l |= __shfl_xor_sync(FULL, m0l, o);
            m0h |= __shfl_xor_sync(FULL, m0h, o);
            m1l |= __shfl_xor_sync(FULL, m1l, o);
            m1h |= __shfl_xor_sync(FULL, m1h, o);
        }
        if ((lane & 3) == 0) {
            if (r0 < n) { dom[2 * r0] = m0l; dom[2 * r0 + 1] = m0h; }
            if (r1 < n) { dom[2 * r1] = m1l; dom[2 * r1 + 1] = m1h; }
        }
        __syncwarp();
    }
    // equal adjacent keys collapse to one
    u64 lo = 0, hi = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const u64 b = __ballot_sync(FULL, i < n && (i == 0 || ck[i] != ck[i - 1]));
        if (i0 < 64) lo |= b << i0; else hi |= b << (i0 - 64);
    }
    int nout = 0;
    const int R = (int)d.R;
    while (nout < R && (lo | hi)) {
        const int head = lo ? __ffsll((long long)lo) - 1 : 64 + __ffsll((long long)hi) - 1;
        if (head < 64) lo &= lo - 1; else hi &= hi - 1;
        if (lane == 0) {
            const u64 hk = ck[head];
            out_id[nout] = key_id(hk);
            out_rho[nout] = key_rho(hk);
        }
        nout++;
        lo &= ~dom[2 * head];
        hi &= ~dom[2 * head + 1];
    }
    __syncwarp();
    return nout;
}

// ---------------------------------------------------------------------------
// RobustPrune over n candidates whose keys ck[0..n) are sorted ascending
// (rho = distance to the owner).  Equal adjacent keys collapse to one.  The
// head is kept; every later candidate p' with alpha^2 * d(head, p') <= rho(p')
// is dropped; stop at R.  Distances between candidates are canonical
// distances, 8 lanes per distance, rows taken from the stage when staged.
// Scratch: alive[n], idx[n].
// ---------------------------------------------------------------------------
// GV, the Gram variant of a kernel: 0, a buffer of at most GRAM_N rows with
// rows of one 128-column block; 1, more than GRAM_N rows (the large path,
// which restages each block per stripe); 2, at most GRAM_N rows spanning
// several blocks (partial sums kept between blocks).
template <int GV>
__device__ int warp_prune(const Dev &d, const u64 *ck, int n, unsigned char *alive, u32 *idx, u32 *out_id,
                          float *out_rho, Stage &st) {
    if (st.gram && n <= st.gram_rows) {
        if constexpr (GV == 1) return warp_prune_masks<GRAM_NL / 8>(d, ck, n, out_id, out_rho, st);
        else return warp_prune_gram<GV == 2>(d, ck, n, alive, out_id, out_rho, st);
    }
    const int lane = lane_id();
    const int grp = lane >> 3, g = lane & 7;
    const int ns = st.rows ? min(n, st.ns_cap) : 0;
    stage_rows(d, st, ck, ns);
    for (int i = lane; i < n; i += 32) alive[i] = (i == 0 || ck[i] != ck[i - 1]) ? 1 : 0;
    __syncwarp();
    auto row = [&](int i) -> const float * {
        return i < ns ? st.rows + (size_t)i * d.mp : d.x + (size_t)key_id(ck[i]) * d.mp;
    };
    int nout = 0, start = 0;
    const int R = (int)d.R;
    while (nout < R) {
        int head = -1;
        for (int i0 = start; i0 < n; i0 += 32) {
            int i = i0 + lane;
            u32 m = __ballot_sync(FULL, i < n && alive[i]);
            if (m) { head = i0 + __ffs(m) - 1; break; }
        }
        if (head < 0) break;
        const u64 hk = ck[head];
        if (lane == 0) { out_id[nout] = key_id(hk); out_rho[nout] = key_rho(hk); }
        nout++;
        if (nout == R) break;
        int m_cnt = 0;
        for (int i0 = head + 1; i0 < n; i0 += 32) {
            int i = i0 + lane;
            bool ok = i < n && alive[i];
            u32 m = __ballot_sync(FULL, ok);
            if (ok) idx[m_cnt + __popc(m & lanemask_lt())] = (u32)i;
            m_cnt += __popc(m);
        }
        __syncwarp();
        const float *hrow = row(head);
        if (d.mp <= 128) {
            // the head's four float4 per lane stay in registers
            float4 hr[4];
            canon_row_q8(hrow, (int)d.mp, g, hr);
            for (int r0 = 0; r0 < m_cnt; r0 += 4) {
                const int c = r0 + grp;
                const int cc = c < m_cnt ? c : m_cnt - 1;
                const u32 j = idx[cc];
                const u64 kj = ck[j];
                float4 v[4];
                canon_row_q8(row((int)j), (int)d.mp, g, v);
                const float dd = canon_dist_q8v(hr, v, (int)d.mp, (int)d.metric, g);
                if (c < m_cnt && g == 0 && __fmul_rn(d.alpha2, dd) <= key_rho(kj)) alive[j] = 0;
            }
        } else {
            for (int r0 = 0; r0 < m_cnt; r0 += 4) {
                const int c = r0 + grp;
                const int cc = c < m_cnt ? c : m_cnt - 1;
                const u32 j = idx[cc];
                const u64 kj = ck[j];
                float dd = canon_dist<8>(hrow, row((int)j), (int)d.mp, (int)d.metric, g);
                if (c < m_cnt && g == 0 && __fmul_rn(d.alpha2, dd) <= key_rho(kj)) alive[j] = 0;
            }
        }
        __syncwarp();
        start = head + 1;
    }
    __syncwarp();
    return nout;
}

// Load N(u) into shared memory; returns the degree and the snapshot word.
__device__ __forceinline__ int load_list(const Dev &d, u32 u, u32 *ids, float *rho, u64 &snap) {
    const int lane = lane_id();
    u64 r = 0;
    if (lane == 0) r = ld_ref(d, u);
    r = __shfl_sync(FULL, r, 0);
    snap = r;
    const u32 s = ref_slab(r);
    const int n = s == NIL ? 0 : (int)ref_deg(r);
    for (int j = lane; j < n; j += 32) {
        uint2 e = d.slab[(size_t)s * d.R + j];
        ids[j] = e.x;
        rho[j] = __uint_as_float(e.y);
    }
    __syncwarp();
    return n;
}

__device__ __forceinline__ bool warp_same_list(const u32 *a, const float *ar, int na, const u32 *b,
                                               const float *br, int nb) {
    if (na != nb) return false;
    const int lane = lane_id();
    bool diff = false;
    for (int j = lane; j < na; j += 32)
        diff |= (a[j] != b[j]) || (__float_as_uint(ar[j]) != __float_as_uint(br[j]));
    return __ballot_sync(FULL, diff) == 0;
}

__device__ __forceinline__ bool warp_contains(const u32 *ids, int n, u32 v) {
    bool hit = false;
    for (int j = lane_id(); j < n; j += 32) hit |= ids[j] == v;
    return __ballot_sync(FULL, hit) != 0;
}

// Apply one offer (v, rho) to the list in place (Algorithm 2, reverse edge):
// a present id is a no-op; below R the entry is inserted in (rho, id) order;
// at R the list is RobustPrune(list + v) about the owner (tombstones drop).
// Scratch: keys[np], alive[np], idx[np] with np >= R + 1 (power of two).
template <int GV>
// pruned: in, whether the list is a RobustPrune output (no entry dropped by
// an earlier one, see ref_pruned); out, the same for the returned list.
__device__ int apply_offer(const Dev &d, u32 *ids, float *rho, int n, u32 v, float vr, u64 *keys,
                           unsigned char *alive, u32 *idx, int np, u32 *oid, float *orho, Stage &st, bool &pruned) {
    const int lane = lane_id();
    if (warp_contains(ids, n, v)) return n;
    const u64 kv = mkkey(vr, v);
    if (n < (int)d.R) {
        pruned = false;   // a plain insertion: v is not checked against the entries
        int pos = 0;
        for (int j0 = 0; j0 < n; j0 += 32) {
            int j = j0 + lane;
            pos += __popc(__ballot_sync(FULL, j < n && mkkey(rho[j], ids[j]) < kv));
        }
        u32 tid[2];
        float tr[2];
        int c = 0;
        for (int j = pos + lane; j < n; j += 32, c++) { tid[c] = ids[j]; tr[c] = rho[j]; }
        __syncwarp();
        c = 0;
        for (int j = pos + lane; j < n; j += 32, c++) { ids[j + 1] = tid[c]; rho[j + 1] = tr[c]; }
        if (lane == 0) { ids[pos] = v; rho[pos] = vr; }
        __syncwarp();
        return n + 1;
    }
    // the list is sorted by (rho, id) and holds no v: the candidates in order
    // are its live entries with v placed at its rank
    int nl = 0, below = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        u64 k = KEY_INF;
        bool live = false;
        if (i < n) {
            k = mkkey(rho[i], ids[i]);
            live = !ref_del(ld_ref(d, ids[i]));
        }
        const u32 lm = __ballot_sync(FULL, live);
        const int pos = nl + __popc(lm & lanemask_lt()) + (k > kv ? 1 : 0);
        if (live) keys[pos] = k;
        below += __popc(__ballot_sync(FULL, live && k < kv));
        nl += __popc(lm);
    }
    // A full list of live entries that no earlier entry drops, with v after
    // all of them: the prune keeps the R entries in order and stops before v.
    st.wk_state += 8ull * n;                 // the entries' reference words
    if (pruned && nl == n && below == nl) return n;
    if (lane == 0) keys[below] = kv;
    __syncwarp();
    const int cn = nl + 1;
    st.wk_rows += prune_row_bytes(d, st, cn);
    int nout = warp_prune<GV>(d, keys, cn, alive, idx, oid, orho, st);
    for (int j = lane; j < nout; j += 32) { ids[j] = oid[j]; rho[j] = orho[j]; }
    __syncwarp();
    pruned = true;
    return nout;
}

// ---------------------------------------------------------------------------
// Forward edges: F_v = RobustPrune(C_v) with C_v the expanded non-tombstone
// nodes of v's search (nearest max_cand); Publish(v, F_v); emit offers.
// ---------------------------------------------------------------------------
struct PruneInsArgs {
    Dev d;
    u32 first, b;
    const u64 *exp_keys;
    const u32 *exp_count;
    u32 max_hops, max_cand, np, ns, gram;
    u32 rescore;   // the search ran on a reduced-precision copy: rescore in fp32
    u32 *F_id;
    float *F_rho;
    u32 *F_n;
    Offers of;
};

__host__ __device__ inline size_t prune_ins_scratch(u32 np, u32 R) {
    return al16(np) + al16((size_t)np * 4) + 2 * al16((size_t)R * 4);
}
__host__ __device__ inline size_t prune_ins_warp_bytes(u32 np, u32 R, u32 ns, u32 mp, u32 gram) {
    const size_t sc = prune_ins_scratch(np, R);
    return stage_bytes(ns, mp) + al16((size_t)np * 8) + (gram_alias(gram, sc) ? 0 : sc) + gram_bytes(gram, mp);
}

// one-warp blocks (the launch uses 32 threads); the small-path instantiation
// is held to 12 resident warps per SM (at most 170 registers a thread)
template <int GV>
__global__ void __launch_bounds__(32, GV == 1 ? 1 : 12) prune_insert_kernel(PruneInsArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const u32 R = d.R;
    char *p = smem + warp * prune_ins_warp_bytes(a.np, R, a.ns, d.mp, a.gram);
    char *gbuf = a.gram ? p : nullptr;
    p += gram_bytes(a.gram, d.mp);
    Stage st = stage_init(p, a.ns, d.mp, gbuf, a.gram);
    WarpSlabs ws;
    ws_init(ws);
    p += stage_bytes(a.ns, d.mp);
    u64 *keys = reinterpret_cast<u64 *>(p); p += al16((size_t)a.np * 8);
    if (gram_alias(a.gram, prune_ins_scratch(a.np, R))) p = gbuf;
    unsigned char *alive = reinterpret_cast<unsigned char *>(p); p += al16(a.np);
    u32 *idx = reinterpret_cast<u32 *>(p); p += al16((size_t)a.np * 4);
    u32 *oid = reinterpret_cast<u32 *>(p); p += al16((size_t)R * 4);
    float *orho = reinterpret_cast<float *>(p);
    u32 t_next = 0;   // the next item's claim, in flight while this one runs
    if (lane == 0) t_next = (u32)atomicAdd(&d.ctr[C_WORK], 1ull);
    for (;;) {
        const u32 t = __shfl_sync(FULL, t_next, 0);
        if (t >= a.b) break;
        if (lane == 0) t_next = (u32)atomicAdd(&d.ctr[C_WORK], 1ull);
        const u32 cnt = a.exp_count[t];
        for (u32 i = lane; i < a.np; i += 32) keys[i] = i < cnt ? a.exp_keys[(size_t)t * a.max_hops + i] : KEY_INF;
        __syncwarp();
        warp_sort_u64(keys, (int)a.np);
        const int n = (int)min(cnt, a.max_cand);
        const u32 v = dev_first(d, a.first) + t;
        if (a.rescore) {
            // the nearest max_cand by the search's reduced-precision distance,
            // re-scored with the canonical fp32 distance to v and re-sorted,
            // so that RobustPrune and every stored rho see exact distances
            const float *xv = d.x + (size_t)v * d.mp;
            const int grp = lane >> 3, g = lane & 7;
            for (int r0 = 0; r0 < n; r0 += 4) {
                const int c = min(r0 + grp, n - 1);
                const u32 id = key_id(keys[c]);
                const float dist = canon_dist<8>(xv, d.x + (size_t)id * d.mp, (int)d.mp, (int)d.metric, g);
                __syncwarp();
                if (r0 + grp < n && g == 0) keys[c] = mkkey(dist, id);
                __syncwarp();
            }
            for (u32 i = n + lane; i < a.np; i += 32) keys[i] = KEY_INF;
            __syncwarp();
            warp_sort_u64(keys, (int)a.np);
        }
        // rows: the candidates (fp32 for the re-score, with v's own row)
        st.wk_rows += a.rescore ? (u64)(n + 1) * 4 * d.mp : prune_row_bytes(d, st, n);
        const int nout = warp_prune<GV>(d, keys, n, alive, idx, oid, orho, st);
        u64 snap = 0;
        if (lane == 0) snap = ld_ref(d, v);
        snap = __shfl_sync(FULL, snap, 0);
        st.wk_state += 8 + 8ull * nout + 8;     // v's word read, its list and word written
        if (!warp_publish(d, ws, v, oid, orho, nout, snap, true) && lane == 0)
            atomicOr(&d.ctr[C_ERR], (u64)ERR_CAS);
        const u32 invalid = (u32)d.capacity;
        for (u32 j = lane; j < R; j += 32) {
            const size_t o = (size_t)t * R + j;
            const bool ok = (int)j < nout;
            a.F_id[o] = ok ? oid[j] : NIL;
            a.F_rho[o] = ok ? orho[j] : 0.0f;
            a.of.key[o] = ok ? oid[j] : invalid;
            a.of.val[o] = (u32)o;
            a.of.src[o] = v;
            a.of.rho[o] = ok ? orho[j] : 0.0f;
        }
        if (lane == 0) a.F_n[t] = (u32)nout;
        __syncwarp();
    }
    ws_finish(d, ws);
    stage_done(d, st, WK_PRUNE);
}

cudaError_t launch_prune_insert(const Dev &d, u32 first, u32 b, const u64 *exp_keys, const u32 *exp_count,
                                u32 max_hops, u32 max_cand, u32 *F_id, float *F_rho, u32 *F_n,
                                const Offers &of, int num_sms, cudaStream_t st, bool rescore) {
    if (b == 0) return cudaSuccess;
    // the Gram tile covers the prune only when every candidate fits in it
    const u32 gram = gram_rows_for(d.gram, max_cand);
    PruneInsArgs a{d, first, b, exp_keys, exp_count, max_hops, max_cand, 0, 0, gram, rescore ? 1u : 0u,
                   F_id, F_rho, F_n, of};
    u32 np = 32;
    while (np < max_hops) np <<= 1;
    a.np = np;
    a.ns = gram ? 0 : stage_cap(d.mp, max_cand, d.stage_bytes);
    const size_t wb = prune_ins_warp_bytes(np, d.R, a.ns, d.mp, gram);
    const int W = warps_for(wb);
    size_t smem = W * wb;
    const void *fns[3] = {(const void *)prune_insert_kernel<0>, (const void *)prune_insert_kernel<1>, (const void *)prune_insert_kernel<2>};
    const void *fn = fns[gram_variant(a.gram, d.mp)];
    cudaError_t e = smem_at_least((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, fn, 32 * W, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    u32 blocks = (u32)(per_sm * num_sms), need = (b + W - 1) / W;
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(d.ctr + C_WORK, 0, sizeof(u64), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(blocks), dim3(32 * W), args, smem, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reverse offers.  Deterministic: one warp per target segment, offers in
// ascending source order, one publish.  Lock-free: one warp per offer,
// CAS-published with retries up to `budget` (Algorithm 1).
// ---------------------------------------------------------------------------
struct FoldArgs {
    Dev d;
    Offers of;
    const u32 *seg_start;
    const u64 *seg_count;
    u32 budget;   // 0 = deterministic
    u32 np, ns, gram;
    u32 lo, hi;   // lock-free: offer slots [lo, hi) of this launch
};

__host__ __device__ inline size_t fold_scratch(u32 np, u32 R) {
    return 2 * al16((size_t)R * 4 + 4) + al16(np) + al16((size_t)np * 4);
}
// keys: a prune sees at most R + 1 candidates
__host__ __device__ inline size_t fold_warp_bytes(u32 np, u32 R, u32 ns, u32 mp, u32 gram) {
    const size_t sc = fold_scratch(np, R);
    return stage_bytes(ns, mp) + 4 * al16((size_t)R * 4 + 4) + al16((size_t)(R + 1) * 8) +
           (gram_alias(gram, sc) ? 0 : sc) + gram_bytes(gram, mp);
}

// one-warp blocks (the launch uses 32 threads); the small-path instantiation
// is held to 12 resident warps per SM (at most 170 registers a thread)
template <int GV>
__global__ void __launch_bounds__(32, GV == 1 ? 1 : 12) offer_fold_kernel(FoldArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const u32 R = d.R;
    char *p = smem + warp * fold_warp_bytes(a.np, R, a.ns, d.mp, a.gram);
    char *gbuf = a.gram ? p : nullptr;
    p += gram_bytes(a.gram, d.mp);
    Stage st = stage_init(p, a.ns, d.mp, gbuf, a.gram);
    WarpSlabs ws;
    ws_init(ws);
    p += stage_bytes(a.ns, d.mp);
    const size_t lb = al16((size_t)R * 4 + 4);
    u32 *lid = reinterpret_cast<u32 *>(p); p += lb;
    float *lrho = reinterpret_cast<float *>(p); p += lb;
    u32 *oid0 = reinterpret_cast<u32 *>(p); p += lb;
    float *orho0 = reinterpret_cast<float *>(p); p += lb;
    u64 *keys = reinterpret_cast<u64 *>(p); p += al16((size_t)(R + 1) * 8);
    if (gram_alias(a.gram, fold_scratch(a.np, R))) p = gbuf;
    u32 *tid = reinterpret_cast<u32 *>(p); p += lb;
    float *trho = reinterpret_cast<float *>(p); p += lb;
    unsigned char *alive = reinterpret_cast<unsigned char *>(p); p += al16(a.np);
    u32 *idx = reinterpret_cast<u32 *>(p);
    const u64 nwork = a.budget ? (u64)(a.hi - a.lo) : *a.seg_count;
    u64 t_next = 0;   // the next item's claim, in flight while this one runs
    if (lane == 0) t_next = atomicAdd(&d.ctr[C_WORK], 1ull);
    u64 pf_t = ~0ull;   // lock-free: the item whose words pf_w, pf_v, pf_vr hold
    u32 pf_w = 0, pf_v = 0;
    float pf_vr = 0.f;
    for (;;) {
        const u64 t = __shfl_sync(FULL, t_next, 0);
        if (t >= nwork) break;
        if (lane == 0) t_next = atomicAdd(&d.ctr[C_WORK], 1ull);
        if (a.budget == 0) {
            const u32 lo = a.seg_start[t], hi = a.seg_start[t + 1];
            const u32 w = a.of.key[lo];
            u64 snap;
            const int n0 = load_list(d, w, lid, lrho, snap);
            st.wk_state += 8 + 8ull * n0;
            for (int j = lane; j < n0; j += 32) { oid0[j] = lid[j]; orho0[j] = lrho[j]; }
            __syncwarp();
            int n = n0;
            bool pruned = ref_pruned(snap) != 0;
            for (u32 q = lo; q < hi; q++) {
                const u32 pi = a.of.val[q];
                n = apply_offer<GV>(d, lid, lrho, n, a.of.src[pi], a.of.rho[pi], keys, alive, idx, (int)a.np,
                                tid, trho, st, pruned);
            }
            if (!warp_same_list(lid, lrho, n, oid0, orho0, n0)) {
                st.wk_state += 8ull * n + 8;
                if (!warp_publish(d, ws, w, lid, lrho, n, snap, pruned) && lane == 0)
                    atomicOr(&d.ctr[C_ERR], (u64)ERR_CAS);
            }
        } else {
            u32 w = pf_w, v = pf_v;
            float vr = pf_vr;
            if (t != pf_t) { w = a.of.key[t + a.lo]; v = a.of.src[t + a.lo]; vr = a.of.rho[t + a.lo]; }
            if (w >= (u32)d.capacity) continue;
            bool done = false;
            for (u32 att = 0; att < a.budget && !done; att++) {
                u64 snap;
                const int n0 = load_list(d, w, lid, lrho, snap);
                st.wk_state += 8 + 8ull * n0;
                for (int j = lane; j < n0; j += 32) { oid0[j] = lid[j]; orho0[j] = lrho[j]; }
                __syncwarp();
                bool pruned = ref_pruned(snap) != 0;
                const int n = apply_offer<GV>(d, lid, lrho, n0, v, vr, keys, alive, idx, (int)a.np, tid, trho, st,
                                              pruned);
                if (att == 0) {                      // the next offer's words, in flight while this one publishes
                    pf_t = __shfl_sync(FULL, t_next, 0);
                    if (pf_t < nwork) { pf_w = a.of.key[pf_t + a.lo]; pf_v = a.of.src[pf_t + a.lo]; pf_vr = a.of.rho[pf_t + a.lo]; }
                }
                if (warp_same_list(lid, lrho, n, oid0, orho0, n0)) { done = true; break; }
                st.wk_state += 8ull * n + 8;
                done = warp_publish(d, ws, w, lid, lrho, n, snap, pruned);
                u64 err = 0;
                if (lane == 0) err = *reinterpret_cast<volatile u64 *>(&d.ctr[C_ERR]);
                if (!done && (__shfl_sync(FULL, err, 0) & ERR_NOMEM)) break;
            }
            if (!done && lane == 0) atomicAdd(&d.ctr[C_DROPPED], 1ull);
        }
        __syncwarp();
    }
    ws_finish(d, ws);
    stage_done(d, st, WK_OFFER);
}

cudaError_t launch_offer_fold(const Dev &d, const Offers &of, const u32 *seg_start, const u64 *seg_count,
                              u32 budget, int num_sms, cudaStream_t st, u32 lo, u32 hi) {
    if (of.n == 0) return cudaSuccess;
    if (budget && hi > of.n) hi = of.n;
    if (budget && lo >= hi) return cudaSuccess;
    FoldArgs a{d, of, seg_start, seg_count, budget, 0, 0, gram_rows_for(d.gram, d.R + 1), lo, budget ? hi : of.n};
    u32 np = 32;
    while (np < d.R + 1) np <<= 1;
    a.np = np;
    a.ns = d.gram ? 0 : stage_cap(d.mp, d.R + 1, d.stage_bytes);
    const size_t wb = fold_warp_bytes(np, d.R, a.ns, d.mp, a.gram);
    const int W = warps_for(wb);
    size_t smem = W * wb;
    const void *fns[3] = {(const void *)offer_fold_kernel<0>, (const void *)offer_fold_kernel<1>, (const void *)offer_fold_kernel<2>};
    const void *fn = fns[gram_variant(a.gram, d.mp)];
    cudaError_t e = smem_at_least((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, fn, 32 * W, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const u32 items = budget ? a.hi - a.lo : of.n;
    u32 blocks = (u32)(per_sm * num_sms), need = (items + W - 1) / W;
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(d.ctr + C_WORK, 0, sizeof(u64), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(blocks), dim3(32 * W), args, smem, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Refine pass (reading of Sec. 3.4.1): member v re-selects its edges from
// N(v) and the lists of its neighbours (two hops; mode 2 admits only members
// of the same sub-batch), keeps the nearest max_cand, prunes, publishes if
// the list changed, and offers the edges it gained.
// ---------------------------------------------------------------------------
struct RefineArgs {
    Dev d;
    u32 first, b, mode, max_cand, cap, np, ns, gram;
    u32 cap_s, np_s;   // the shared-memory lists (most members); cap, np: the full ones
    char *spill;       // per warp, lists for cap raw ids (a member with more)
    u64 spill_warp;    // bytes of one warp's spill lists
    Offers of;
};

// Bytes of one warp's candidate lists for `cap` raw two-hop ids.
__host__ __device__ inline size_t refine_list_bytes(u32 np, u32 cap) {
    return al16((size_t)np * 8) + al16(np) + al16((size_t)np * 4) + al16((size_t)cap * 4);
}

__host__ __device__ inline size_t refine_warp_bytes(u32 np, u32 cap, u32 R, u32 ns, u32 mp, u32 gram) {
    return stage_bytes(ns, mp) + 4 * al16((size_t)R * 4) + refine_list_bytes(np, cap) + gram_bytes(gram, mp);
}

template <int GV>
__global__ void __launch_bounds__(64, GV == 1 ? 1 : 6) refine_kernel(RefineArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const u32 R = d.R;
    char *p = smem + warp * refine_warp_bytes(a.np_s, a.cap_s, R, a.ns, d.mp, a.gram);
    char *gbuf = a.gram ? p : nullptr;
    p += gram_bytes(a.gram, d.mp);
    Stage st = stage_init(p, a.ns, d.mp, gbuf, a.gram);
    WarpSlabs ws;
    ws_init(ws);
    p += stage_bytes(a.ns, d.mp);
    u32 *nid = reinterpret_cast<u32 *>(p); p += al16((size_t)R * 4);
    float *nrho = reinterpret_cast<float *>(p); p += al16((size_t)R * 4);
    u32 *oid = reinterpret_cast<u32 *>(p); p += al16((size_t)R * 4);
    float *orho = reinterpret_cast<float *>(p); p += al16((size_t)R * 4);
    // lists: in shared memory for up to cap_s raw ids, else this warp's spill
    auto carve_lists = [](char *q, u32 np) {
        struct L { u64 *buf; unsigned char *alive; u32 *idx, *uid; } l;
        l.buf = reinterpret_cast<u64 *>(q); q += al16((size_t)np * 8);
        l.alive = reinterpret_cast<unsigned char *>(q); q += al16(np);
        l.idx = reinterpret_cast<u32 *>(q); q += al16((size_t)np * 4);
        l.uid = reinterpret_cast<u32 *>(q);
        return l;
    };
    const auto ls = carve_lists(p, a.np_s);
    const auto lg = carve_lists(a.spill + (blockIdx.x * (blockDim.x >> 5) + warp) * a.spill_warp, a.np);
    const int grp = lane >> 3, g = lane & 7;
    u32 t_next = 0;   // the next item's claim, in flight while this one runs
    if (lane == 0) t_next = (u32)atomicAdd(&d.ctr[C_WORK], 1ull);
    for (;;) {
        const u32 t = __shfl_sync(FULL, t_next, 0);
        if (t >= a.b) break;
        if (lane == 0) t_next = (u32)atomicAdd(&d.ctr[C_WORK], 1ull);
        const u32 v = dev_first(d, a.first) + t;
        u64 snap;
        const int dv = load_list(d, v, nid, nrho, snap);
        st.wk_state += 8 + 8ull * dv;
        // 1. raw two-hop ids (v, members of N(v), and for mode 2 non-members
        //    of the sub-batch excluded), kept as u64 for the sort; a member
        //    with more than cap_s of them is collected again into the spill
        u64 *buf = ls.buf;
        unsigned char *alive = ls.alive;
        u32 *idx = ls.idx, *uid = ls.uid;
        u32 cap = a.cap_s;
        int nraw = 0;
        bool overflow = false;
        u64 nb_state = 0;                       // the neighbours' words and lists
    collect:
        nraw = 0;
        overflow = false;
        nb_state = 0;
        for (int i = 0; i < dv; i++) {
            const u64 rw = ld_ref(d, nid[i]);
            const u32 s = ref_slab(rw);
            const int dw = s == NIL ? 0 : (int)ref_deg(rw);
            nb_state += 8 + 8ull * dw;
            for (int j0 = 0; j0 < dw; j0 += 32) {
                u32 y = NIL;
                if (j0 + lane < dw) y = d.slab[(size_t)s * R + j0 + lane].x;
                bool ok = y != NIL && y != v;
                if (ok && a.mode == 2) ok = y >= dev_first(d, a.first) && y < dev_first(d, a.first) + a.b;
                if (ok) {
                    for (int k = 0; k < dv; k++) ok &= nid[k] != y;
                }
                u32 m = __ballot_sync(FULL, ok);
                int pos = nraw + __popc(m & lanemask_lt());
                if (ok) {
                    if (pos < (int)cap) buf[pos] = y;
                    else overflow = true;
                }
                nraw += __popc(m);
            }
        }
        if (__any_sync(FULL, overflow)) {
            if (buf == ls.buf) {
                buf = lg.buf;
                alive = lg.alive;
                idx = lg.idx;
                uid = lg.uid;
                cap = a.cap;
                goto collect;
            }
            if (lane == 0) atomicOr(&d.ctr[C_ERR], (u64)ERR_OVERFLOW);
            nraw = min(nraw, (int)a.cap);
        }
        st.wk_state += nb_state;
        int np2 = 32;
        while (np2 < nraw) np2 <<= 1;
        for (int i = nraw + lane; i < np2; i += 32) buf[i] = KEY_INF;
        __syncwarp();
        warp_sort_u64(buf, np2);
        // 2. unique live ids
        int nu = 0;
        for (int i0 = 0; i0 < nraw; i0 += 32) {
            int i = i0 + lane;
            bool ok = i < nraw && (i == 0 || buf[i] != buf[i - 1]);
            u32 y = ok ? (u32)buf[i] : NIL;
            if (ok && a.mode != 2) ok = !ref_del(ld_ref(d, y));
            u32 m = __ballot_sync(FULL, ok);
            if (ok) uid[nu + __popc(m & lanemask_lt())] = y;
            nu += __popc(m);
        }
        __syncwarp();
        // 3. distances to v, then the live members of N(v)
        st.wk_rows += (u64)(nu + 1) * 4 * d.mp;   // v's row and the peers'
        st.wk_state += 8ull * ((a.mode != 2 ? nu : 0) + dv);   // liveness words
        const float *vrow = d.x + (size_t)v * d.mp;
        if (d.mp <= 128) {
            // v's four float4 per lane stay in registers
            float4 vr[4];
            canon_row_q8(vrow, (int)d.mp, g, vr);
            for (int r0 = 0; r0 < nu; r0 += 4) {
                const int c = r0 + grp;
                const int cc = c < nu ? c : nu - 1;
                const u32 y = uid[cc];
                float4 w4[4];
                canon_row_q8(d.x + (size_t)y * d.mp, (int)d.mp, g, w4);
                const float dd = canon_dist_q8v(vr, w4, (int)d.mp, (int)d.metric, g);
                if (c < nu && g == 0) buf[c] = mkkey(dd, y);
            }
        } else {
            for (int r0 = 0; r0 < nu; r0 += 4) {
                const int c = r0 + grp;
                const int cc = c < nu ? c : nu - 1;
                const u32 y = uid[cc];
                float dd = canon_dist<8>(vrow, d.x + (size_t)y * d.mp, (int)d.mp, (int)d.metric, g);
                if (c < nu && g == 0) buf[c] = mkkey(dd, y);
            }
        }
        __syncwarp();
        int nc = nu;
        for (int j0 = 0; j0 < dv; j0 += 32) {
            int j = j0 + lane;
            bool ok = j < dv && !ref_del(ld_ref(d, nid[j]));
            u32 m = __ballot_sync(FULL, ok);
            if (ok) buf[nc + __popc(m & lanemask_lt())] = mkkey(nrho[j], nid[j]);
            nc += __popc(m);
        }
        // The re-selection cannot change a pruned list of live entries (see
        // ref_pruned) when no peer was found, or when the list is full and
        // every peer sorts after it: the prune keeps the list in order.
        bool same = false;
        if (ref_pruned(snap) && nc - nu == dv) {
            const u64 last = dv ? mkkey(nrho[dv - 1], nid[dv - 1]) : 0ull;
            bool early = false;
            for (int i = lane; i < nu; i += 32) early |= buf[i] < last;
            same = nu == 0 || (dv == (int)R && !__any_sync(FULL, early));
        }
        int nout = dv;
        if (same) {
            for (int j = lane; j < dv; j += 32) { oid[j] = nid[j]; orho[j] = nrho[j]; }
            __syncwarp();
        } else {
            int np3 = 32;
            while (np3 < nc) np3 <<= 1;
            for (int i = nc + lane; i < np3; i += 32) buf[i] = KEY_INF;
            __syncwarp();
            warp_sort_u64(buf, np3);
            const int n = min(nc, (int)a.max_cand);
            st.wk_rows += prune_row_bytes(d, st, nc - nu);   // the members of N(v), not yet gathered
            nout = warp_prune<GV>(d, buf, n, alive, idx, oid, orho, st);
            if (!warp_same_list(oid, orho, nout, nid, nrho, dv)) {
                st.wk_state += 8ull * nout + 8;
                if (!warp_publish(d, ws, v, oid, orho, nout, snap, true) && lane == 0)
                    atomicOr(&d.ctr[C_ERR], (u64)ERR_CAS);
            }
        }
        const u32 invalid = (u32)d.capacity;
        for (u32 j = lane; j < R; j += 32) {
            const size_t o = (size_t)t * R + j;
            bool gained = false;
            if ((int)j < nout) {
                gained = true;
                for (int k = 0; k < dv; k++) gained &= nid[k] != oid[j];
            }
            a.of.key[o] = gained ? oid[j] : invalid;
            a.of.val[o] = (u32)o;
            a.of.src[o] = v;
            a.of.rho[o] = gained ? orho[j] : 0.0f;
        }
        __syncwarp();
    }
    ws_finish(d, ws);
    stage_done(d, st, WK_REFINE);
}

// Launch shape of the refine kernel (shared by launch_refine and the spill size).
static void refine_shape(const Dev &d, u32 max_cand, RefineArgs &a) {
    u32 cap = d.R * d.R;
    if (cap > 4096) cap = 4096;
    a.cap = cap;
    u32 np = 32;
    while (np < cap + d.R) np <<= 1;
    a.np = np;
    a.cap_s = cap < 192u ? cap : 192u;
    u32 nps = 32;
    while (nps < a.cap_s + d.R) nps <<= 1;
    a.np_s = nps;
    a.gram = d.gram ? (d.R > 32 ? (u32)GRAM_NL : (u32)GRAM_N) : 0u;
    a.ns = d.gram ? 0 : stage_cap(d.mp, max_cand, d.stage_bytes);
    a.spill_warp = refine_list_bytes(np, cap);
}

size_t refine_spill_bytes(const Dev &d, u32 max_cand, int num_sms) {
    RefineArgs a{};
    refine_shape(d, max_cand, a);
    // every warp an SM can hold (2,048 threads)
    return (size_t)num_sms * 64 * a.spill_warp;
}

cudaError_t launch_refine(const Dev &d, u32 first, u32 b, u32 mode, u32 max_cand, const Offers &of,
                          int num_sms, cudaStream_t st, char *spill, size_t spill_bytes) {
    if (b == 0) return cudaSuccess;
    RefineArgs a;
    a.d = d; a.first = first; a.b = b; a.mode = mode; a.max_cand = max_cand; a.of = of;
    refine_shape(d, max_cand, a);
    a.spill = spill;
    const size_t wb = refine_warp_bytes(a.np_s, a.cap_s, d.R, a.ns, d.mp, a.gram);
    const int warps = 2 * wb <= 200 * 1024 ? 2 : 1;
    size_t smem = warps * wb;
    const void *fns[3] = {(const void *)refine_kernel<0>, (const void *)refine_kernel<1>, (const void *)refine_kernel<2>};
    const void *fn = fns[gram_variant(a.gram, d.mp)];
    cudaError_t e = smem_at_least((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, fn, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    u32 blocks = (u32)(per_sm * num_sms), need = (b + warps - 1) / warps;
    if (blocks > need) blocks = need;
    if ((size_t)blocks * warps * a.spill_warp > spill_bytes) return cudaErrorInvalidValue;
    e = cudaMemsetAsync(d.ctr + C_WORK, 0, sizeof(u64), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(blocks), dim3(32 * warps), args, smem, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Delete: tombstone CAS <0,d,s> -> <1,d,s> over ids sorted ascending; a
// repeated, unknown, already deleted or reclaimed id is a no-op.
// ---------------------------------------------------------------------------
__global__ void tombstone_kernel(Dev d, const u32 *ids, u32 n, u64 next_id, u32 *ok) {
    u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32 u = ids[i];
    u32 res = 0;
    if ((i == 0 || ids[i - 1] != u) && (u64)u < dev_next_id(d, next_id)) {
        for (int att = 0; att < 64; att++) {
            const u64 r = ld_ref(d, u);
            if (ref_del(r) || ref_slab(r) == NIL) break;
            if (atomicCAS(&d.ref[u], r, r | (1ull << 63)) == r) { res = 1; break; }
        }
    }
    ok[i] = res;
}

cudaError_t launch_tombstone(const Dev &d, const u32 *sorted_ids, u32 n, u64 next_id, u32 *ok, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    tombstone_kernel<<<(n + 255) / 256, 256, 0, st>>>(d, sorted_ids, n, next_id, ok);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Repair, step 1: for deleted u with B = N(u) and each live a in B,
// K(u, a) = RobustPrune_a(B \ {a}).  The distances among B are computed once
// per u into a table; the prune reads the table.
// ---------------------------------------------------------------------------
struct RepairKArgs {
    Dev d;
    const u32 *dt;
    const u64 *n_dt;
    u32 max_n, ns, gram;
    u32 *pair_key, *pair_val;
    uint2 *pair_K;
    u32 *pair_Kn;
};

// sort width for K: the warp bitonic sort needs a power of two >= 32
__host__ __device__ inline u32 repk_np(u32 R) {
    u32 np = 32;
    while (np < R) np <<= 1;
    return np;
}

__host__ __device__ inline size_t repk_warp_bytes(u32 R, u32 ns, u32 mp, u32 gram) {
    const u32 np = repk_np(R);
    return stage_bytes(ns, mp) + 2 * al16((size_t)R * 4) + al16((size_t)R * R * 4) + al16((size_t)32 * np + 32) +
           gram_bytes(gram, mp);
}

__global__ void __launch_bounds__(128, 1) repair_k_kernel(RepairKArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const u32 R = d.R;
    char *p = smem + warp * repk_warp_bytes(R, a.ns, d.mp, a.gram);
    char *gbuf = a.gram ? p : nullptr;
    p += gram_bytes(a.gram, d.mp);
    Stage st = stage_init(p, a.ns, d.mp, gbuf, a.gram);
    p += stage_bytes(a.ns, d.mp);
    u32 *bid = reinterpret_cast<u32 *>(p); p += al16((size_t)R * 4);
    u32 *bdel = reinterpret_cast<u32 *>(p); p += al16((size_t)R * 4);
    float *M = reinterpret_cast<float *>(p); p += al16((size_t)R * R * 4);
    const int npk = (int)repk_np(R);
    unsigned char *ord = reinterpret_cast<unsigned char *>(p) + lane * npk;   // this lane's sorted candidates
    const int grp = lane >> 3, g = lane & 7;
    const u64 nd = *a.n_dt;
    const u32 invalid = (u32)d.capacity;
    u64 i_next = 0;   // the next item's claim, in flight while this one runs
    if (lane == 0) i_next = atomicAdd(&d.ctr[C_WORK], 1ull);
    for (;;) {
        const u64 i = __shfl_sync(FULL, i_next, 0);
        if (i >= nd) break;
        if (lane == 0) i_next = atomicAdd(&d.ctr[C_WORK], 1ull);
        const u32 u = a.dt[i];
        u64 r = 0;
        if (lane == 0) r = ld_ref(d, u);
        r = __shfl_sync(FULL, r, 0);
        const u32 s = ref_slab(r);
        const int nb = s == NIL ? 0 : (int)ref_deg(r);
        for (int j = lane; j < nb; j += 32) {
            bid[j] = d.slab[(size_t)s * R + j].x;
            bdel[j] = ref_del(ld_ref(d, bid[j]));
        }
        st.wk_state += 8 + 16ull * nb;           // u's word, N(u), and the members' words
        st.wk_rows += (u64)nb * 4 * d.mp;        // B's rows (the canonical table)
        __syncwarp();
        // distance table among B (symmetric).  These distances become the
        // stored rho of replacement edges, so they stay canonical.
        const int nsb = st.rows ? min(nb, st.ns_cap) : 0;
        stage_rows_by(d, st, nsb, [&](int i) { return bid[i]; });
        auto brow = [&](int i) -> const float * {
            return i < nsb ? st.rows + (size_t)i * d.mp : d.x + (size_t)bid[i] * d.mp;
        };
        // the pairs x < y in one sequence (index y (y - 1) / 2 + x), eight per
        // trip in two independent rounds of four: their row loads overlap
        const int npair = nb * (nb - 1) / 2;
        auto pair_of = [](int q, int &x, int &y) {
            int yy = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)q)) * 0.5f);
            if (yy * (yy - 1) / 2 > q) yy--;
            if ((yy + 1) * yy / 2 <= q) yy++;
            y = yy;
            x = q - yy * (yy - 1) / 2;
        };
        if (d.mp <= 128) {
            // rows of at most 128 floats: each lane's four float4 of both rows
            // of a pair in registers, so the canonical distance runs with no
            // column loop; each group's pair cursor steps by 8 in the same
            // sequence instead of recomputing it with a square root
            int x = 0, y = 1, x2 = 0, y2 = 1;
            if (grp < npair) pair_of(grp, x, y);
            if (grp + 4 < npair) pair_of(grp + 4, x2, y2);
            for (int q0 = 0; q0 < npair; q0 += 8) {
                const int q = q0 + grp, q2 = q + 4;
                const bool v1 = q < npair, v2 = q2 < npair;
                float4 ra[4], rb[4], rc[4], rd[4];
                canon_row_q8(brow(v1 ? x : 0), (int)d.mp, g, ra);
                canon_row_q8(brow(v1 ? y : 1), (int)d.mp, g, rb);
                canon_row_q8(brow(v2 ? x2 : 0), (int)d.mp, g, rc);
                canon_row_q8(brow(v2 ? y2 : 1), (int)d.mp, g, rd);
                const float dd = canon_dist_q8v(ra, rb, (int)d.mp, (int)d.metric, g);
                const float dd2 = canon_dist_q8v(rc, rd, (int)d.mp, (int)d.metric, g);
                if (v1 && g == 0) { M[x * R + y] = dd; M[y * R + x] = dd; }
                if (v2 && g == 0) { M[x2 * R + y2] = dd2; M[y2 * R + x2] = dd2; }
                for (x += 8; x >= y; y++) x -= y;
                for (x2 += 8; x2 >= y2; y2++) x2 -= y2;
            }
        } else {
            for (int q0 = 0; q0 < npair; q0 += 8) {
                const int q = q0 + grp, q2 = q + 4;
                int x, y, x2, y2;
                pair_of(q < npair ? q : npair - 1, x, y);
                pair_of(q2 < npair ? q2 : npair - 1, x2, y2);
                const float dd = canon_dist<8>(brow(x), brow(y), (int)d.mp, (int)d.metric, g);
                const float dd2 = canon_dist<8>(brow(x2), brow(y2), (int)d.mp, (int)d.metric, g);
                if (q < npair && g == 0) { M[x * R + y] = dd; M[y * R + x] = dd; }
                if (q2 < npair && g == 0) { M[x2 * R + y2] = dd2; M[y2 * R + x2] = dd2; }
            }
        }
        __syncwarp();
        // K(u, a) for every a in B, one lane per a: the candidates b != a, live,
        // in ascending (d(a, b), b), then the greedy RobustPrune on the table.
        // Orders: with |B| <= 32 the warp sorts each a's candidates in
        // registers (the id replaced by its rank among B's ids: the same
        // order, and the rank leads back to the table index); above that each
        // lane ranks its own candidates by counting.
        u32 liveB = 0;
        for (int t0 = 0; t0 < nb; t0 += 32) {
            const u32 m = __ballot_sync(FULL, t0 + lane < nb && !bdel[t0 + lane]);
            if (t0 == 0) liveB = m;
        }
        const bool sorted_by_warp = nb <= 32;
        if (sorted_by_warp) {
            int idr = 0;
            if (lane < nb)
                for (int t2 = 0; t2 < nb; t2++) idr += bid[t2] < bid[lane];
            unsigned char *inv = reinterpret_cast<unsigned char *>(ord) - lane * npk + 32 * npk;   // after the orders
            if (lane < nb) inv[idr] = (unsigned char)lane;
            __syncwarp();
            for (int ja0 = 0; ja0 < nb; ja0 += 4) {
                u64 k[4];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int ja = ja0 + c;
                    const bool v = ja < nb && (liveB >> ja & 1) && lane < nb && lane != ja && (liveB >> lane & 1);
                    k[c] = v ? ((u64)f2ord(M[ja * R + lane]) << 32) | (u32)idr : KEY_INF;   // M is symmetric
                }
                warp_sort32x4(k);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    unsigned char *oa = reinterpret_cast<unsigned char *>(ord) - lane * npk + (ja0 + c) * npk;
                    if (k[c] != KEY_INF) oa[lane] = inv[(u32)k[c]];
                }
            }
            __syncwarp();
        }
        for (int ja = lane; ja < (int)R; ja += 32) {
            const size_t slot = (size_t)i * R + ja;
            if (ja >= nb || bdel[ja]) {
                a.pair_key[slot] = invalid;
                a.pair_val[slot] = (u32)slot;
                a.pair_Kn[slot] = 0;
                continue;
            }
            int nc = 0;
            if (sorted_by_warp) {
                nc = __popc(liveB & ~(1u << ja));
            } else {
                // rank of each candidate among the candidates (keys are distinct: ids
                // differ); M is symmetric, and M[t][ja] keeps the lanes on distinct banks
                for (int t = 0; t < nb; t++) {
                    if (t == ja || bdel[t]) continue;
                    const u64 kt = mkkey(M[t * R + ja], bid[t]);
                    int rank = 0;
                    for (int t2 = 0; t2 < nb; t2++)
                        if (t2 != ja && !bdel[t2] && mkkey(M[t2 * R + ja], bid[t2]) < kt) rank++;
                    ord[rank] = (unsigned char)t;
                    nc++;
                }
            }
            int nk = 0;
            u64 alive = nc >= 64 ? ~0ull : ((1ull << nc) - 1);
            for (int h = 0; h < nc && nk < (int)R; h++) {
                if (!(alive >> h & 1)) continue;
                const int hj = ord[h];
                const float hr = M[hj * R + ja];
                a.pair_K[slot * R + nk] = make_uint2(bid[hj], __float_as_uint(hr));
                nk++;
                for (int t2 = h + 1; t2 < nc; t2++) {
                    if (!(alive >> t2 & 1)) continue;
                    const int tj = ord[t2];
                    if (__fmul_rn(d.alpha2, M[hj * R + tj]) <= M[tj * R + ja]) alive &= ~(1ull << t2);
                }
            }
            a.pair_key[slot] = bid[ja];
            a.pair_val[slot] = (u32)slot;
            a.pair_Kn[slot] = (u32)nk;
        }
        __syncwarp();
    }
    stage_done(d, st, WK_REPAIR_K);
}

cudaError_t launch_repair_k(const Dev &d, const u32 *dt, const u64 *n_dt, u32 max_n, u32 *pair_key,
                            u32 *pair_val, uint2 *pair_K, u32 *pair_Kn, int num_sms, cudaStream_t st) {
    if (max_n == 0) return cudaSuccess;
    // B's rows are read about |B| times each: stage up to 16 KB of them
    const u32 budget = d.stage_bytes > (16u << 10) ? d.stage_bytes : (16u << 10);
    RepairKArgs a{d, dt, n_dt, max_n, stage_cap(d.mp, d.R, budget), 0u, pair_key, pair_val, pair_K, pair_Kn};
    const size_t wb = repk_warp_bytes(d.R, a.ns, d.mp, a.gram);
    const int W = warps_for(wb);
    size_t smem = W * wb;
    cudaError_t e = smem_at_least((const void *)repair_k_kernel, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, repair_k_kernel, 32 * W, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    u32 blocks = (u32)(per_sm * num_sms), need = (max_n + W - 1) / W;
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(d.ctr + C_WORK, 0, sizeof(u64), st);
    if (e != cudaSuccess) return e;
    repair_k_kernel<<<blocks, 32 * W, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Repair, step 2: for each live a, in ascending u:
// N <- RobustPrune_a((N \ {u}) + K(u, a)); publish once if changed.
// Lock-free mode (seg_start == NULL): one warp per (u, a) pair, CAS retries.
// ---------------------------------------------------------------------------
struct RepairFoldArgs {
    Dev d;
    const u32 *dt, *pair_key, *pair_val;
    const uint2 *pair_K;
    const u32 *pair_Kn;
    const u32 *seg_start;
    const u64 *seg_count;
    u64 n_pairs;
    u32 budget, np, ns, gram;
    u64 lo;       // lock-free: pair slots [lo, lo + n_pairs) of this launch
};

__host__ __device__ inline size_t repf_scratch(u32 np, u32 R) {
    return 2 * al16((size_t)R * 4 + 4) + 2 * al16((size_t)np * 8) + al16(np) + al16((size_t)np * 4);
}
__host__ __device__ inline size_t repf_warp_bytes(u32 np, u32 R, u32 ns, u32 mp, u32 gram) {
    const size_t sc = repf_scratch(np, R);
    return stage_bytes(ns, mp) + 4 * al16((size_t)R * 4 + 4) + al16((size_t)np * 8) +
           (gram_alias(gram, sc) ? 0 : sc) + gram_bytes(gram, mp);
}

template <int GV>
// pruned: in, whether the list is a RobustPrune output (see ref_pruned);
// out, the same for the returned list.
__device__ int repair_apply(const Dev &d, u32 *lid, float *lrho, int n, u32 u, const uint2 *K, int nk, u64 *keys,
                            u64 *ka, u64 *kb, unsigned char *alive, u32 *idx, int np, u32 *tid, float *trho,
                            Stage &st, bool &pruned) {
    const int lane = lane_id();
    // The list (minus u and deleted nodes) and K(u, a) (minus deleted nodes)
    // are each sorted by (rho, id); compact both, then place every key at its
    // rank in the union: a K key after the list keys below it, a list key after
    // the K keys below it.  An id in both has equal keys and would collapse in
    // the prune; its K copy is dropped here (same result, fewer Gram rows).
    int na = 0, nb = 0;
    uint2 e0 = make_uint2(0u, 0u);                   // K's first 32 entries, in flight with the list's words
    if (lane < nk) e0 = K[lane];
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const bool v = i < n && lid[i] != u && !ref_del(ld_ref(d, lid[i]));
        const u32 m = __ballot_sync(FULL, v);
        if (v) ka[na + __popc(m & lanemask_lt())] = mkkey(lrho[i], lid[i]);
        na += __popc(m);
    }
    for (int j0 = 0; j0 < nk; j0 += 32) {
        const int j = j0 + lane;
        uint2 e = e0;
        if (j0 > 0 && j < nk) e = K[j];
        const bool v = j < nk && !ref_del(ld_ref(d, e.x));
        const u32 m = __ballot_sync(FULL, v);
        if (v) kb[nb + __popc(m & lanemask_lt())] = mkkey(__uint_as_float(e.y), e.x);
        nb += __popc(m);
    }
    __syncwarp();
    int nb2 = 0;                                     // K keys not in the list, compacted in place
    bool early = false;                              // a kept K key sorts before the list's last key
    for (int j0 = 0; j0 < nb; j0 += 32) {
        const int j = j0 + lane;
        u64 k = 0;
        int lo = 0;
        bool keep = false;
        if (j < nb) {
            k = kb[j];
            int hi = na;                             // list keys <= k
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ka[mid] <= k) lo = mid + 1; else hi = mid;
            }
            keep = lo == 0 || ka[lo - 1] != k;
        }
        const u32 m = __ballot_sync(FULL, keep);
        const int jj = nb2 + __popc(m & lanemask_lt());
        if (keep) { kb[jj] = k; keys[jj + lo] = k; }
        nb2 += __popc(m);
        early |= __ballot_sync(FULL, keep && lo < na) != 0;
    }
    __syncwarp();
    // The list is full, live, without u, and no entry drops a later one; every
    // K key left sorts after it: the prune keeps the R entries in order and
    // stops before the first K key.
    st.wk_state += 8ull * (n + nk);          // reference words of the list and of K(u, a)
    if (pruned && na == n && n == (int)d.R && !early) return n;
    for (int i = lane; i < na; i += 32) {
        const u64 k = ka[i];
        int lo = 0, hi = nb2;                        // kept K keys < k
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (kb[mid] < k) lo = mid + 1; else hi = mid;
        }
        keys[i + lo] = k;
    }
    __syncwarp();
    const int cn = na + nb2;
    st.wk_rows += prune_row_bytes(d, st, cn);
    const int nout = warp_prune<GV>(d, keys, cn, alive, idx, tid, trho, st);
    for (int j = lane; j < nout; j += 32) { lid[j] = tid[j]; lrho[j] = trho[j]; }
    __syncwarp();
    pruned = true;
    return nout;
}

// one-warp blocks (the launch uses 32 threads); the small-path instantiation
// is held to 12 resident warps per SM (at most 170 registers a thread)
template <int GV>
__global__ void __launch_bounds__(32, GV == 1 ? 1 : 12) repair_fold_kernel(RepairFoldArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const u32 R = d.R;
    char *p = smem + warp * repf_warp_bytes(a.np, R, a.ns, d.mp, a.gram);
    char *gbuf = a.gram ? p : nullptr;
    p += gram_bytes(a.gram, d.mp);
    Stage st = stage_init(p, a.ns, d.mp, gbuf, a.gram);
    WarpSlabs ws;
    ws_init(ws);
    p += stage_bytes(a.ns, d.mp);
    const size_t lb = al16((size_t)R * 4 + 4);
    u32 *lid = reinterpret_cast<u32 *>(p); p += lb;
    float *lrho = reinterpret_cast<float *>(p); p += lb;
    u32 *oid0 = reinterpret_cast<u32 *>(p); p += lb;
    float *orho0 = reinterpret_cast<float *>(p); p += lb;
    u64 *keys = reinterpret_cast<u64 *>(p); p += al16((size_t)a.np * 8);
    if (gram_alias(a.gram, repf_scratch(a.np, R))) p = gbuf;
    u32 *tid = reinterpret_cast<u32 *>(p); p += lb;
    float *trho = reinterpret_cast<float *>(p); p += lb;
    u64 *ka = reinterpret_cast<u64 *>(p); p += al16((size_t)a.np * 8);
    u64 *kb = reinterpret_cast<u64 *>(p); p += al16((size_t)a.np * 8);
    unsigned char *alive = reinterpret_cast<unsigned char *>(p); p += al16(a.np);
    u32 *idx = reinterpret_cast<u32 *>(p);
    const u64 nwork = a.budget ? a.n_pairs : *a.seg_count;
    u64 t_next = 0;   // the next item's claim, in flight while this one runs
    if (lane == 0) t_next = atomicAdd(&d.ctr[C_WORK], 1ull);
    u64 pf_t = ~0ull;   // lock-free: the item whose words pf_w, pf_pv hold
    u32 pf_w = 0, pf_pv = 0;
    for (;;) {
        const u64 t = __shfl_sync(FULL, t_next, 0);
        if (t >= nwork) break;
        if (lane == 0) t_next = atomicAdd(&d.ctr[C_WORK], 1ull);
        if (a.budget == 0) {
            const u32 lo = a.seg_start[t], hi = a.seg_start[t + 1];
            const u32 w = a.pair_key[lo];
            u64 snap;
            const int n0 = load_list(d, w, lid, lrho, snap);
            st.wk_state += 8 + 8ull * n0;
            for (int j = lane; j < n0; j += 32) { oid0[j] = lid[j]; orho0[j] = lrho[j]; }
            __syncwarp();
            int n = n0;
            bool pruned = ref_pruned(snap) != 0;
            for (u32 q = lo; q < hi; q++) {
                const u32 pv = a.pair_val[q];
                n = repair_apply<GV>(d, lid, lrho, n, a.dt[pv / R], a.pair_K + (size_t)pv * R, (int)a.pair_Kn[pv], keys,
                                 ka, kb, alive, idx, (int)a.np, tid, trho, st, pruned);
            }
            if (!warp_same_list(lid, lrho, n, oid0, orho0, n0)) {
                st.wk_state += 8ull * n + 8;
                if (!warp_publish(d, ws, w, lid, lrho, n, snap, pruned) && lane == 0)
                    atomicOr(&d.ctr[C_ERR], (u64)ERR_CAS);
            }
        } else {
            u32 w = pf_w, pv = pf_pv;
            if (t != pf_t) { w = a.pair_key[t + a.lo]; pv = a.pair_val[t + a.lo]; }
            if (w >= (u32)d.capacity) continue;
            bool done = false;
            for (u32 att = 0; att < a.budget && !done; att++) {
                u64 snap;
                const int n0 = load_list(d, w, lid, lrho, snap);
                st.wk_state += 8 + 8ull * n0;
                for (int j = lane; j < n0; j += 32) { oid0[j] = lid[j]; orho0[j] = lrho[j]; }
                __syncwarp();
                bool pruned = ref_pruned(snap) != 0;
                const int n = repair_apply<GV>(d, lid, lrho, n0, a.dt[pv / R], a.pair_K + (size_t)pv * R,
                                           (int)a.pair_Kn[pv], keys, ka, kb, alive, idx, (int)a.np, tid, trho, st,
                                           pruned);
                if (att == 0) {                      // the next pair's words, in flight while this one publishes
                    pf_t = __shfl_sync(FULL, t_next, 0);
                    if (pf_t < nwork) { pf_w = a.pair_key[pf_t + a.lo]; pf_pv = a.pair_val[pf_t + a.lo]; }
                }
                if (warp_same_list(lid, lrho, n, oid0, orho0, n0)) { done = true; break; }
                st.wk_state += 8ull * n + 8;
                done = warp_publish(d, ws, w, lid, lrho, n, snap, pruned);
                u64 err = 0;
                if (lane == 0) err = *reinterpret_cast<volatile u64 *>(&d.ctr[C_ERR]);
                if (!done && (__shfl_sync(FULL, err, 0) & ERR_NOMEM)) break;
            }
            if (!done && lane == 0) atomicAdd(&d.ctr[C_DROPPED], 1ull);
        }
        __syncwarp();
    }
    ws_finish(d, ws);
    stage_done(d, st, WK_REPAIR_FOLD);
}

cudaError_t launch_repair_fold(const Dev &d, const u32 *dt, const u32 *pair_key, const u32 *pair_val,
                                    const uint2 *pair_K, const u32 *pair_Kn, const u32 *seg_start,
                                    const u64 *seg_count, u64 n_pairs, u32 budget, int num_sms, cudaStream_t st,
                               u64 lo) {
    if (n_pairs == 0) return cudaSuccess;
    RepairFoldArgs a{d, dt, pair_key, pair_val, pair_K, pair_Kn, seg_start, seg_count, n_pairs, budget, 0, 0,
                     gram_rows_for(d.gram, 2 * d.R - 1), lo};
    u32 np = 32;
    while (np < 2 * d.R) np <<= 1;
    a.np = np;
    a.ns = d.gram ? 0 : stage_cap(d.mp, 2 * d.R, d.stage_bytes);
    const size_t wb = repf_warp_bytes(np, d.R, a.ns, d.mp, a.gram);
    const int W = warps_for(wb);
    size_t smem = W * wb;
    const void *fns[3] = {(const void *)repair_fold_kernel<0>, (const void *)repair_fold_kernel<1>, (const void *)repair_fold_kernel<2>};
    const void *fn = fns[gram_variant(a.gram, d.mp)];
    cudaError_t e = smem_at_least((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, fn, 32 * W, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    u64 need = (n_pairs + W - 1) / W;
    u32 blocks = (u32)(per_sm * num_sms);
    if ((u64)blocks > need) blocks = (u32)need;
    e = cudaMemsetAsync(d.ctr + C_WORK, 0, sizeof(u64), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(blocks), dim3(32 * W), args, smem, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Reclaim phase 1 (compaction): every live node with a tombstoned neighbour
// republishes its list without those entries, order and rho kept.  One warp
// per 32 consecutive ids; tombstones are read from a bitmap.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) compact_kernel(Dev d, u64 next_id, const u32 *tomb_bits) {
    __shared__ u32 sid[8][MAX_R];
    __shared__ float srho[8][MAX_R];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const u64 base = ((u64)blockIdx.x * 8 + warp) * 32;
    next_id = dev_next_id(d, next_id);
    if (base >= next_id) return;
    const u64 myid = base + lane;
    const u64 myref = myid < next_id ? ld_ref(d, (u32)myid) : ref_pack(1, 0, NIL);
    const u32 R = d.R;
    WarpSlabs ws;
    ws_init(ws);
    // graph state: the words scanned, each live list with one tombstone bit
    // per entry, and the lists republished
    u64 wk = 8ull * (u64)min((u64)32, next_id - base);
    for (int t = 0; t < 32; t++) {
        const u64 r = __shfl_sync(FULL, myref, t);
        if (ref_del(r) || ref_slab(r) == NIL) continue;
        const u32 s = ref_slab(r);
        const int n = (int)ref_deg(r);
        wk += 8ull * n + (u64)(n + 7) / 8;
        bool dirty = false;
        u32 ids[2];
        float rhos[2];
        bool keep[2];
        int c = 0;
        for (int j = lane; j < n; j += 32, c++) {
            uint2 e = d.slab[(size_t)s * R + j];
            ids[c] = e.x;
            rhos[c] = __uint_as_float(e.y);
            const bool dead = (tomb_bits[e.x >> 5] >> (e.x & 31)) & 1u;
            keep[c] = !dead;
            dirty |= dead;
        }
        if (!__any_sync(FULL, dirty)) continue;
        int nk = 0;
        c = 0;
        for (int j0 = 0; j0 < n; j0 += 32, c++) {
            const int j = j0 + lane;
            const bool k = j < n && keep[c];
            const u32 m = __ballot_sync(FULL, k);
            if (k) { sid[warp][nk + __popc(m & lanemask_lt())] = ids[c]; srho[warp][nk + __popc(m & lanemask_lt())] = rhos[c]; }
            nk += __popc(m);
        }
        __syncwarp();
        // a lost CAS here means another writer touched the node during the
        // reclaim launch, which the launch discipline forbids
        wk += 8ull * nk + 8;
        if (!warp_publish(d, ws, (u32)(base + t), sid[warp], srho[warp], nk, r, ref_pruned(r) != 0) && lane == 0)
            atomicOr(&d.ctr[C_ERR], (u64)ERR_CAS);
        __syncwarp();
    }
    ws_finish(d, ws);
    if (lane == 0) atomicAdd(&d.ctr[C_WK + 2 * WK_COMPACT + 1], wk);
}

cudaError_t launch_compact(const Dev &d, u64 next_id, const u32 *tomb_bits, cudaStream_t st) {
    if (next_id == 0) return cudaSuccess;
    u64 warps = (next_id + 31) / 32;
    compact_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(d, next_id, tomb_bits);
    return cudaGetLastError();
}

// Reclaim phase 2: CAS <1,d,s> -> <1,0,NIL> and retire s.
__global__ void reclaim_tomb_kernel(Dev d, u64 next_id) {
    const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= dev_next_id(d, next_id)) return;
    const u64 r = ld_ref(d, (u32)u);
    if (!ref_del(r) || ref_slab(r) == NIL) return;
    if (atomicCAS(&d.ref[u], r, ref_pack(1, 0, NIL)) == r) retire_slab(d, ref_slab(r));
    else atomicOr(&d.ctr[C_ERR], (u64)ERR_CAS);
}

cudaError_t launch_reclaim_tombstones(const Dev &d, u64 next_id, cudaStream_t st) {
    if (next_id == 0) return cudaSuccess;
    reclaim_tomb_kernel<<<(unsigned)((next_id + 255) / 256), 256, 0, st>>>(d, next_id);
    return cudaGetLastError();
}

}  // namespace etale
