// search.cu — BeamSearch (Sec. 3.4.1) for inserts and queries, one warp per
// query, persistent grid fed by an atomic work counter.
//
// Per expansion the warp reads the expanded node's slab (the reference word
// was read when the node entered the beam), drops neighbours it has already
// evaluated, gathers the remaining neighbour rows into shared memory with
// bulk (TMA) copies completing on an mbarrier, computes their canonical
// distances with 8 lanes per distance, and merges them into the beam.
//
// Visited set.  The beam semantics are those of an exact visited set: an id
// evaluated once is never evaluated again.  The kernel keeps only a lossy
// direct-mapped cache of evaluated ids (no false positives) and, when the
// cache misses, may evaluate an id a second time.  That changes nothing:
// once the beam is full its worst key only decreases, so an id that left the
// beam or was refused is refused again (its key is the same), and an id still
// in the beam is recognised in the merge by its equal key and dropped.
#include <algorithm>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "internal.h"

namespace etale {

struct SearchArgs {
    Dev d;
    const float *q;      // query rows, stride mp floats, 16-byte aligned
    const u64 *seed;     // nq x L initial beams (top-L of the entry set), KEY_INF padded
    const u32 *nq_dev;   // when set, the batch size is read here (CUDA graphs); nq is its cap
    u32 nq, L, max_hops, mode;   // mode 0: query, 1: insert
    u32 k;
    u32 *out_ids;
    float *out_dist;
    u64 *exp_keys;       // insert: nq x max_hops expanded non-tombstone keys
    u32 *exp_count;
    u32 stage_rows, seen_slots, seen_bits;
    // the evaluated-id cache (see seen_layout): 0 = whole ids, else 8- or
    // 16-bit tags behind a validity bitmap of seen_words words
    u32 seen_tag, seen_shift, seen_tmask, seen_hmask, seen_words;
    u32 rowb;            // bytes per gathered row (fp32, bf16 or fp8 copy)
    u32 wq, err;         // work-queue counter and error word (query searches
                         // use their own, so they can overlap a writer)
    u32 rerank;          // reduced precision: re-scored candidates (<= 64)
    u32 exact;           // P = 1 over a bf16 copy that holds every row exactly: no rerank
    u32 rekey;           // P != 0 with seeds ranked in fp32: re-key them in P and re-sort
    u32 tc;              // P = 1 reduced-precision search: keys from tensor-core dot products (tc_keys)
    u32 srow;            // stage row stride in bytes (rowb, or padded for the tensor-core path)
    u32 *elog;           // diagnostic (LOG kernels): per query, the ids evaluated during
    u32 *elog_n;         //   expansions in order (elog_cap slots) and their count
    u32 elog_cap;
};

// Row gathered for a neighbour: the fp32 row or its reduced-precision copy.
template <int P>
__device__ __forceinline__ const void *row_src(const Dev &d, u32 id) {
    if (P == 1) return d.xb + (size_t)id * d.mb;
    if (P == 2) return d.x8 + (size_t)id * d.m8;
    return d.x + (size_t)id * d.mp;
}

// Four dequantised elements [i, i + 4) of a staged row.
template <int P>
__device__ __forceinline__ float4 load4(const void *row, int i, float scale) {
    if (P == 1) {
        const uint2 w = *reinterpret_cast<const uint2 *>(reinterpret_cast<const unsigned short *>(row) + i);
        return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xFFFF0000u),
                           __uint_as_float(w.y << 16), __uint_as_float(w.y & 0xFFFF0000u));
    } else if (P == 2) {
        const unsigned int w = *reinterpret_cast<const unsigned int *>(reinterpret_cast<const unsigned char *>(row) + i);
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
        return make_float4(__fmul_rn(a.x, scale), __fmul_rn(a.y, scale), __fmul_rn(b.x, scale), __fmul_rn(b.y, scale));
    } else {
        return *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(row) + i);
    }
}

// The canonical reduction tree (see canon_dist) over a row of precision P,
// G lanes per distance (lane g of the group holds partials g, g + G, ...):
// fp32 arithmetic on dequantised values.  Every G gives the same value.
template <int P, int G>
__device__ __forceinline__ float qdist_g(const float *__restrict__ q, const void *row, float scale, int mp, int metric,
                                         int g) {
    if (P == 0) return canon_dist<G>(q, reinterpret_cast<const float *>(row), mp, metric, g);
    constexpr int T = 32 / G;
    float p[T];
#pragma unroll
    for (int t = 0; t < T; t++) {
        const int j = g + G * t;
        float acc = 0.0f;
        for (int base = 0; base < mp; base += 128) {
            const int i = base + 4 * j;
            if (i < mp) {
                const float4 u = *reinterpret_cast<const float4 *>(q + i);
                const float4 v = load4<P>(row, i, scale);
                if (metric == 0) {
                    float d0 = __fsub_rn(u.x, v.x), d1 = __fsub_rn(u.y, v.y);
                    float d2 = __fsub_rn(u.z, v.z), d3 = __fsub_rn(u.w, v.w);
                    acc = __fmaf_rn(d0, d0, acc);
                    acc = __fmaf_rn(d1, d1, acc);
                    acc = __fmaf_rn(d2, d2, acc);
                    acc = __fmaf_rn(d3, d3, acc);
                } else {
                    acc = __fmaf_rn(u.x, v.x, acc);
                    acc = __fmaf_rn(u.y, v.y, acc);
                    acc = __fmaf_rn(u.z, v.z, acc);
                    acc = __fmaf_rn(u.w, v.w, acc);
                }
            }
        }
        p[t] = acc;
    }
#pragma unroll
    for (int hh = T / 2; hh >= 1; hh >>= 1)
#pragma unroll
        for (int t = 0; t < hh; t++) p[t] = __fadd_rn(p[t], p[t + hh]);
    float s = p[0];
#pragma unroll
    for (int h = G / 2; h >= 1; h >>= 1) s = __fadd_rn(s, __shfl_xor_sync(FULL, s, h));
    return metric == 0 ? s : __fsub_rn(1.0f, s);
}

// 8 lanes per distance (the staged search and seeding steps).
template <int P>
__device__ __forceinline__ float qdist(const float *__restrict__ q, const void *row, float scale, int mp, int metric,
                                       int g) {
    return qdist_g<P, 8>(q, row, scale, mp, metric, g);
}

// canon_dist<8> for rows of at most 128 floats with this lane's four query
// float4 (elements 4 (g + 8 t) .. + 3, t = 0..3; zero past the row) held in
// registers: the same operations in the same order.
__device__ __forceinline__ float canon_dist_q8(const float4 (&qr)[4], const float *__restrict__ b, int mp, int metric,
                                               int g) {
    float p[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int i = 4 * (g + 8 * t);
        float acc = 0.0f;
        if (i < mp) {
            const float4 u = qr[t];
            const float4 v = *reinterpret_cast<const float4 *>(b + i);
            if (metric == 0) {
                float d0 = __fsub_rn(u.x, v.x), d1 = __fsub_rn(u.y, v.y);
                float d2 = __fsub_rn(u.z, v.z), d3 = __fsub_rn(u.w, v.w);
                acc = __fmaf_rn(d0, d0, acc);
                acc = __fmaf_rn(d1, d1, acc);
                acc = __fmaf_rn(d2, d2, acc);
                acc = __fmaf_rn(d3, d3, acc);
            } else {
                acc = __fmaf_rn(u.x, v.x, acc);
                acc = __fmaf_rn(u.y, v.y, acc);
                acc = __fmaf_rn(u.z, v.z, acc);
                acc = __fmaf_rn(u.w, v.w, acc);
            }
        }
        p[t] = acc;
    }
    p[0] = __fadd_rn(p[0], p[2]);
    p[1] = __fadd_rn(p[1], p[3]);
    float s = __fadd_rn(p[0], p[1]);
#pragma unroll
    for (int h = 4; h >= 1; h >>= 1) s = __fadd_rn(s, __shfl_xor_sync(FULL, s, h));
    return metric == 0 ? s : __fsub_rn(1.0f, s);
}

struct WarpSmem {
    float *qv;       // mp
    float *stage;    // stage_rows x mp
    u64 *bkey;       // beam keys (L), ascending
    u64 *bref;       // reference word sampled when the entry was evaluated
    unsigned char *bflag;   // expanded flag
    u64 *nkey;       // 32: surviving new keys, sorted
    u64 *nref;       // 32
    u32 *cid;        // 32 candidate ids
    u64 *ckey;       // 32
    u64 *cref;       // 32
    u32 *seen;       // seen_slots
    u64 *bar;        // mbarrier; with tensor-core keys, |bf16(q)|^2 (bar + 16 bytes) and
                     // the query as bf16 pairs (bar + 32 bytes) follow it (tc_nq, tc_qb)
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Layout of a warp's evaluated-id cache of 2^bits slots.  With ids below
// 2^cb (cb >= bits, from the capacity), h = id * 2654435761 mod 2^cb is a
// bijection of [0, 2^cb); slot = h >> (cb - bits) and tag = the low cb - bits
// bits of h identify the id, so a slot need only hold the tag: 8 or 16 bits
// when cb - bits allows, beside one validity bit per slot.  Otherwise the
// slot holds the whole id (slot = the top bits of the 32-bit product).  A
// hit is therefore never wrong; a slot overwritten by another id only costs
// a repeated evaluation.
struct SeenLayout {
    u32 tag, shift, tmask, hmask, words;
    size_t bytes;
};
inline SeenLayout seen_layout(u64 capacity, u32 bits) {
    u32 cb = bits;
    while (cb < 32 && (1ull << cb) < capacity) cb++;
    SeenLayout l;
    l.shift = cb - bits;
    l.tag = l.shift <= 8 ? 8u : l.shift <= 16 ? 16u : 0u;
    l.tmask = (1u << l.shift) - 1u;
    l.hmask = cb >= 32 ? ~0u : (1u << cb) - 1u;
    const size_t slots = (size_t)1 << bits;
    l.words = (u32)(slots >= 32 ? slots / 32 : 1);
    l.bytes = l.tag == 0 ? slots * 4 : (size_t)l.words * 4 + slots * (l.tag / 8);
    return l;
}

// srow: stage row stride in bytes; qbytes: the bf16 query of the tensor-core keys (or 0)
__host__ __device__ inline size_t search_warp_bytes(u32 mp, u32 L, u32 stage_rows, size_t seen_bytes, u32 srow,
                                                   u32 qbytes = 0) {
    size_t b = 0;
    b += align_up((size_t)mp * 4, 128);
    b += align_up((size_t)stage_rows * srow, 128);
    b += 2 * align_up((size_t)L * 8, 16);
    b += align_up((size_t)L, 16);
    b += 32 * 8 * 2 + 32 * 4 + 32 * 8 * 2;
    b += align_up(seen_bytes, 16);
    b += 16;
    if (qbytes) b += 16 + align_up(qbytes, 16);
    return align_up(b, 128);
}

__device__ inline WarpSmem carve(char *p, u32 mp, u32 L, u32 stage_rows, size_t seen_bytes, u32 srow,
                                 u32 qbytes = 0) {
    WarpSmem s;
    s.qv = reinterpret_cast<float *>(p); p += align_up((size_t)mp * 4, 128);
    s.stage = reinterpret_cast<float *>(p); p += align_up((size_t)stage_rows * srow, 128);
    s.bkey = reinterpret_cast<u64 *>(p); p += align_up((size_t)L * 8, 16);
    s.bref = reinterpret_cast<u64 *>(p); p += align_up((size_t)L * 8, 16);
    s.bflag = reinterpret_cast<unsigned char *>(p); p += align_up((size_t)L, 16);
    s.nkey = reinterpret_cast<u64 *>(p); p += 32 * 8;
    s.nref = reinterpret_cast<u64 *>(p); p += 32 * 8;
    s.ckey = reinterpret_cast<u64 *>(p); p += 32 * 8;
    s.cref = reinterpret_cast<u64 *>(p); p += 32 * 8;
    s.cid = reinterpret_cast<u32 *>(p); p += 32 * 4;
    s.seen = reinterpret_cast<u32 *>(p); p += align_up(seen_bytes, 16);
    s.bar = reinterpret_cast<u64 *>(p);
    (void)qbytes;
    return s;
}

// The tensor-core keys' query data, laid out after the mbarrier.
__device__ __forceinline__ float *tc_nq(const WarpSmem &s) {
    return reinterpret_cast<float *>(reinterpret_cast<char *>(s.bar) + 16);
}
__device__ __forceinline__ u32 *tc_qb(const WarpSmem &s) {
    return reinterpret_cast<u32 *>(reinterpret_cast<char *>(s.bar) + 32);
}

__device__ __forceinline__ u32 seen_slot(u32 id, u32 bits) { return (id * 2654435761u) >> (32 - bits); }

__host__ __device__ inline size_t seen_bytes(const SearchArgs &a) {
    return a.seen_tag == 0 ? (size_t)a.seen_slots * 4 : (size_t)a.seen_words * 4 + (size_t)a.seen_slots * (a.seen_tag / 8);
}

__device__ __forceinline__ bool seen_has(const SearchArgs &a, const WarpSmem &s, u32 id) {
    if (a.seen_tag == 0) return s.seen[seen_slot(id, a.seen_bits)] == id;
    const u32 h = (id * 2654435761u) & a.seen_hmask, slot = h >> a.seen_shift, tag = h & a.seen_tmask;
    if (!((s.seen[slot >> 5] >> (slot & 31)) & 1u)) return false;
    const void *tags = s.seen + a.seen_words;
    return a.seen_tag == 8 ? reinterpret_cast<const unsigned char *>(tags)[slot] == tag
                           : reinterpret_cast<const unsigned short *>(tags)[slot] == tag;
}

// Lanes may record ids into the same slot at once: one tag stays, its bit set.
__device__ __forceinline__ void seen_put(const SearchArgs &a, const WarpSmem &s, u32 id) {
    if (a.seen_tag == 0) {
        s.seen[seen_slot(id, a.seen_bits)] = id;
        return;
    }
    const u32 h = (id * 2654435761u) & a.seen_hmask, slot = h >> a.seen_shift, tag = h & a.seen_tmask;
    void *tags = s.seen + a.seen_words;
    if (a.seen_tag == 8) reinterpret_cast<unsigned char *>(tags)[slot] = (unsigned char)tag;
    else reinterpret_cast<unsigned short *>(tags)[slot] = (unsigned short)tag;
    atomicOr(s.seen + (slot >> 5), 1u << (slot & 31));
}

__device__ __forceinline__ void seen_clear(const SearchArgs &a, const WarpSmem &s) {
    const u32 n = a.seen_tag == 0 ? a.seen_slots : a.seen_words;
    const u32 v = a.seen_tag == 0 ? NIL : 0u;
    for (u32 i = lane_id(); i < n; i += 32) s.seen[i] = v;
}

__device__ __forceinline__ int lower_bound(const u64 *a, int n, u64 key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Merge the candidate keys held one per lane (KEY_INF = none) into the beam
// in place.  Only keys that can enter the beam take part; entries before the
// first insertion point do not move, so `lo` (every entry before it is
// expanded) drops to that point at most.  Returns the new beam size.
__device__ int merge_beam(WarpSmem &s, u64 key, u64 ref, int n, int L, int &lo) {
    const int lane = lane_id();
    const u64 *bk = s.bkey;
    // drop keys that cannot enter a full beam, and keys already in the beam
    int lb = 0;
    if (key != KEY_INF) {
        if (n == L && key >= bk[n - 1]) {
            key = KEY_INF;
        } else {
            lb = lower_bound(bk, n, key);
            if (lb < n && bk[lb] == key) key = KEY_INF;
        }
    }
    const u32 vm = __ballot_sync(FULL, key != KEY_INF);
    if (vm == 0) return n;
    int rank = 0;
    for (u32 m = vm; m; m &= m - 1) {
        const u64 o = __shfl_sync(FULL, key, __ffs(m) - 1);
        rank += (o < key);
    }
    const int c = __popc(vm);
    if (key != KEY_INF) { s.nkey[rank] = key; s.nref[rank] = ref; }
    // the first insertion point is the lower bound of the smallest new key
    int p0 = (key != KEY_INF && rank == 0) ? lb : 0x7fffffff;
    for (int o = 16; o >= 1; o >>= 1) p0 = min(p0, __shfl_xor_sync(FULL, p0, o));
    lo = min(lo, p0);
    __syncwarp();
    // move entries [p0, n) down, last chunk first so no unread entry is overwritten
    const int nmove = n - p0;
    for (int c0 = ((nmove - 1) >> 5) << 5; c0 >= 0 && nmove > 0; c0 -= 32) {
        const int i = p0 + c0 + lane;
        u64 k2 = 0, r2 = 0;
        unsigned char f2 = 0;
        int pos = 0x7fffffff;
        if (c0 + lane < nmove) {
            k2 = bk[i];
            r2 = s.bref[i];
            f2 = s.bflag[i];
            pos = i + lower_bound(s.nkey, c, k2);   // new keys below it (sorted, distinct)
        }
        __syncwarp();
        if (pos < L) { s.bkey[pos] = k2; s.bref[pos] = r2; s.bflag[pos] = f2; }
        __syncwarp();
    }
    if (key != KEY_INF) {
        const int pos = lb + rank;
        if (pos < L) { s.bkey[pos] = key; s.bref[pos] = ref; s.bflag[pos] = 0; }
    }
    __syncwarp();
    return min(L, n + c);
}

// Tensor-core keys of a reduced-precision BF16 search.  The dot products of
// the bf16 query (s.qb) with the nb <= 32 rows staged at stride a.srow come
// from mma.sync m16n8k16: the query is row 0 of the 16-row A operand, eight
// staged rows at a time are the B operand, read with ldmatrix.  The key is
// |q|^2 + |x|^2 - 2 q.x over the bf16 values (squared L2) or 1 - q.x (inner
// product).  It is one function of (query, id) wherever a key is made in the
// search (neighbours, seeds), so an id evaluated twice has one key.
__device__ void tc_keys(const SearchArgs &a, const WarpSmem &s, int nb, const u32 *ids, u64 *keys) {
    const Dev &d = a.d;
    const int lane = lane_id(), g = lane >> 2, t = lane & 3;
    const u32 sb = smem_addr(s.stage);
    const u32 *qb = tc_qb(s);
    const int ntn = (nb + 7) >> 3;
    const u32 r = lane & 7, mi = lane >> 3;   // the row and the matrix whose address this lane gives
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[nt][c] = 0.0f;
    for (u32 k0 = 0; k0 < d.mb; k0 += 32) {
        // two k-steps of 16; A is zero outside row 0 (lanes 0..3)
        u32 q0 = 0, q1 = 0, q2 = 0, q3 = 0;
        if (g == 0) {
            q0 = qb[(k0 >> 1) + t];
            q1 = qb[(k0 >> 1) + 4 + t];
            q2 = qb[(k0 >> 1) + 8 + t];
            q3 = qb[(k0 >> 1) + 12 + t];
        }
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            if (nt < ntn) {
                u32 row = (u32)nt * 8 + r;
                if ((int)row >= nb) row = 0;   // a staged row; its products are not read
                u32 b0, b1, b2, b3;
                ldsm_x4(b0, b1, b2, b3, sb + row * a.srow + (k0 + 8 * mi) * 2);
                mma_bf16_16816(acc[nt], q0, 0u, q1, 0u, b0, b1);
                mma_bf16_16816(acc[nt], q2, 0u, q3, 0u, b2, b3);
            }
        }
    }
    if (g == 0) {
        const float nq = *tc_nq(s);
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int c = nt * 8 + 2 * t + h;
                if (nt < ntn && c < nb) {
                    const u32 id = ids[c];
                    const float dot = acc[nt][h];
                    const float dist = d.metric == 0 ? __fmaf_rn(-2.0f, dot, __fadd_rn(nq, d.xbn[id]))
                                                     : __fsub_rn(1.0f, dot);
                    keys[c] = mkkey(dist, id);
                }
            }
    }
    __syncwarp();
}

// Bulk-copy the rows of ids[0..nb) (nb <= stage_rows) into the stage at
// stride a.srow and wait for them.
template <int P>
__device__ __forceinline__ void stage_ids(const SearchArgs &a, WarpSmem &s, const u32 *ids, int nb, u32 &phase,
                                          bool &timeout) {
    const int lane = lane_id();
    unsigned char *stage = reinterpret_cast<unsigned char *>(s.stage);
    if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(s.bar, (u32)nb * a.rowb);
    }
    __syncwarp();
    if (lane < nb) bulk_g2s(stage + (size_t)lane * a.srow, row_src<P>(a.d, ids[lane]), a.rowb, s.bar);
    if (!mbar_wait(s.bar, phase, WAIT_LIMIT)) {
        timeout = true;
        mbar_wait(s.bar, phase, WAIT_LIMIT);   // let copies in flight land
    }
    phase ^= 1u;
    __syncwarp();
}

// Evaluate the candidate ids held one per lane (NIL = none) and merge them
// into the beam.  Returns the new beam size.  `phase` tracks the mbarrier.
template <int P, bool LOG>
__device__ int eval_merge(const SearchArgs &a, WarpSmem &s, u32 my_id, int n, u32 &phase, u64 &ndist,
                          bool &timeout, int &lo, const float4 (&qr)[4], u32 *qlog, u32 &qcnt) {
    const Dev &d = a.d;
    const int lane = lane_id();
    const u32 mp = d.mp;
    u32 mask = __ballot_sync(FULL, my_id != NIL);
    const int cnt = __popc(mask);
    if (cnt == 0) return n;
    if (my_id != NIL) s.cid[__popc(mask & lanemask_lt())] = my_id;
    __syncwarp();
    const u32 rowb = a.rowb, srow = P == 1 ? a.srow : a.rowb;   // only BF16 pads its stage rows
    unsigned char *stage = reinterpret_cast<unsigned char *>(s.stage);
    float *scl = reinterpret_cast<float *>(s.nref);   // fp8 scales of the batch (nref is free here)
    for (int b0 = 0; b0 < cnt; b0 += (int)a.stage_rows) {
        const int nb = min((int)a.stage_rows, cnt - b0);
        if (lane == 0) {
            // generic-proxy reads of the stage (previous batch) before async-proxy writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(s.bar, (u32)nb * rowb);
        }
        __syncwarp();
        u64 rf = 0;
        if (lane < nb) {
            const u32 id = s.cid[b0 + lane];
            bulk_g2s(stage + (size_t)lane * srow, row_src<P>(d, id), rowb, s.bar);
            rf = ld_ref(d, id);
            if (P == 2) scl[lane] = d.x8s[id];
        }
        if (!mbar_wait(s.bar, phase, WAIT_LIMIT)) {
            timeout = true;
            mbar_wait(s.bar, phase, WAIT_LIMIT);   // let copies in flight land
        }
        phase ^= 1u;
        if (lane < nb) s.cref[b0 + lane] = rf;
        __syncwarp();
        if (P == 1 && a.tc) {
            tc_keys(a, s, nb, s.cid + b0, s.ckey + b0);
            continue;
        }
        // 8 lanes per distance, 4 distances per round
        const int grp = lane >> 3, g = lane & 7;
        for (int r0 = 0; r0 < nb; r0 += 4) {
            const int c = r0 + grp;
            const int cc = c < nb ? c : nb - 1;   // idle groups recompute a valid row
            float dist;
            if (P == 0 && mp <= 128) {
                dist = canon_dist_q8(qr, reinterpret_cast<const float *>(stage + (size_t)cc * srow), (int)mp,
                                     (int)d.metric, g);
            } else if (P == 1 && mp <= 128) {
                // the bf16 row widened to fp32, then canon_dist's operations in its order
                float4 v[4];
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const int i = 4 * (g + 8 * t);
                    v[t] = i < (int)mp ? load4<1>(stage + (size_t)cc * srow, i, 1.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                dist = canon_dist_q8v(qr, v, (int)mp, (int)d.metric, g);
            } else
                dist = qdist<P>(s.qv, stage + (size_t)cc * srow, P == 2 ? scl[cc] : 1.0f, (int)mp, (int)d.metric, g);
            if (c < nb && g == 0) s.ckey[b0 + c] = mkkey(dist, s.cid[b0 + c]);
        }
        __syncwarp();
    }
    ndist += cnt;
    if (LOG) {
        if (lane < cnt && qcnt + lane < a.elog_cap) qlog[qcnt + lane] = s.cid[lane];
        qcnt += cnt;
    }
    const u64 key = lane < cnt ? s.ckey[lane] : KEY_INF;
    const u64 ref = lane < cnt ? s.cref[lane] : 0;
    if (lane < cnt) seen_put(a, s, key_id(key));
    return merge_beam(s, key, ref, n, (int)a.L, lo);
}

// ---------------------------------------------------------------------------
// Seeding: for each query, the L nearest members of the entry set E by
// (rho, id) (the beam after evaluating every entry point).  A block of 8 warps
// (8 queries) stages 32 entry rows at a time in shared memory; each warp
// computes its 32 distances and merges them into a sorted running top-L.
// ---------------------------------------------------------------------------
constexpr int SEED_TILE = 32;

struct SeedArgs {
    Dev d;
    const float *q;
    const u32 *nq_dev;   // when set, the batch size is read here; nq is its cap
    u32 nq, L;
    u64 *seed;
    u32 rowb;   // bytes per entry row in the tile (fp32 row or its copy)
    const u32 *qsel;     // optional: slot i computes query qsel[i]
};

__host__ __device__ inline size_t seed_warp_bytes(u32 mp, u32 L) {
    return align_up((size_t)mp * 4, 16) + 2 * align_up((size_t)L * 8, 16) + 32 * 8;
}

// In-place merge of the keys held one per lane (KEY_INF = none) into a sorted
// top-L list of keys (the seed kernel's variant of merge_beam: keys only).
__device__ int seed_merge(u64 *bk, u64 *nk, u64 key, int n, int L) {
    const int lane = lane_id();
    int lb = 0;
    if (key != KEY_INF) {
        if (n == L && key >= bk[n - 1]) key = KEY_INF;
        else lb = lower_bound(bk, n, key);
    }
    const u32 vm = __ballot_sync(FULL, key != KEY_INF);
    if (vm == 0) return n;
    int rank = 0;
    for (u32 m = vm; m; m &= m - 1) rank += (__shfl_sync(FULL, key, __ffs(m) - 1) < key);
    const int c = __popc(vm);
    if (key != KEY_INF) nk[rank] = key;
    int p0 = (key != KEY_INF && rank == 0) ? lb : 0x7fffffff;
    for (int o = 16; o >= 1; o >>= 1) p0 = min(p0, __shfl_xor_sync(FULL, p0, o));
    __syncwarp();
    const int nmove = n - p0;
    for (int c0 = ((nmove - 1) >> 5) << 5; c0 >= 0 && nmove > 0; c0 -= 32) {
        const int i = p0 + c0 + lane;
        u64 k2 = 0;
        int pos = 0x7fffffff;
        if (c0 + lane < nmove) {
            k2 = bk[i];
            int cnt = 0;
            for (int j = 0; j < c; j++) cnt += (nk[j] < k2);
            pos = i + cnt;
        }
        __syncwarp();
        if (pos < L) bk[pos] = k2;
        __syncwarp();
    }
    if (key != KEY_INF && lb + rank < L) bk[lb + rank] = key;
    __syncwarp();
    return min(L, n + c);
}

template <int P>
__global__ void __launch_bounds__(256) seed_kernel(SeedArgs a) {
    extern __shared__ __align__(16) char ssm[];
    __shared__ float tscale[SEED_TILE];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const u32 mp = d.mp, L = a.L;
    unsigned char *tile = reinterpret_cast<unsigned char *>(ssm);
    char *p = ssm + align_up((size_t)SEED_TILE * a.rowb, 16) + warp * seed_warp_bytes(mp, L);
    float *qv = reinterpret_cast<float *>(p); p += align_up((size_t)mp * 4, 16);
    u64 *bk0 = reinterpret_cast<u64 *>(p); p += align_up((size_t)L * 8, 16);
    u64 *bk1 = reinterpret_cast<u64 *>(p); p += align_up((size_t)L * 8, 16);
    u64 *nk = reinterpret_cast<u64 *>(p);
    const u32 nq = a.nq_dev ? min(*a.nq_dev, a.nq) : a.nq;
    if (blockIdx.x * 8 >= nq) return;   // block-uniform: no tile work for an empty block
    const u32 slot = blockIdx.x * 8 + warp;
    const bool active = slot < nq;
    const u32 qi = active && a.qsel ? a.qsel[slot] : slot;
    if (active)
        for (u32 i = lane * 4; i < mp; i += 128)
            *reinterpret_cast<float4 *>(qv + i) = *reinterpret_cast<const float4 *>(a.q + (size_t)qi * mp + i);
    const int grp = lane >> 3, g = lane & 7;
    const u32 S = d.nent_dev ? *d.nent_dev : d.n_entries;
    int n = 0;
    for (u32 t0 = 0; t0 < S; t0 += SEED_TILE) {
        const int nt = (int)min((u32)SEED_TILE, S - t0);
        __syncthreads();
        const u32 f4 = a.rowb / 16;
        for (u32 i = threadIdx.x; i < (u32)nt * f4; i += 256) {
            const u32 r = i / f4, c = i % f4;
            reinterpret_cast<uint4 *>(tile + (size_t)r * a.rowb)[c] =
                reinterpret_cast<const uint4 *>(row_src<P>(d, d.entries[t0 + r]))[c];
        }
        if (P == 2 && threadIdx.x < (u32)nt) tscale[threadIdx.x] = d.x8s[d.entries[t0 + threadIdx.x]];
        __syncthreads();
        if (!active) continue;
        u64 key = KEY_INF;
        for (int r0 = 0; r0 < nt; r0 += 4) {
            const int c = r0 + grp;
            const int cc = c < nt ? c : nt - 1;
            const float dist = qdist<P>(qv, tile + (size_t)cc * a.rowb, P == 2 ? tscale[cc] : 1.0f, (int)mp,
                                        (int)d.metric, g);
            const u64 kk = mkkey(dist, d.entries[t0 + cc]);
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const u64 v = __shfl_sync(FULL, kk, t * 8);
                if (lane == r0 + t && r0 + t < nt) key = v;
            }
        }
        n = seed_merge(bk0, nk, key, n, (int)L);
    }
    if (active) {
        for (u32 i = lane; i < L; i += 32) a.seed[(size_t)qi * L + i] = (int)i < n ? bk0[i] : KEY_INF;
    }
}

// One query's BeamSearch by one warp, for slot qi: the query row is
// a.q + qi * mp, the beam starts from the seeds a.seed + qi * L (the L
// nearest entry points, KEY_INF padded, n0 of them valid); query mode writes
// the k results to a.out_ids / a.out_dist + qi * k, insert mode the expanded
// keys of batch member qi.  The reference words of the seeds are sampled here.
template <int P, bool LOG>
__device__ __forceinline__ void search_one(const SearchArgs &a, WarpSmem &s, u32 qi, int n0, u32 &phase,
                                           u64 &nexp_tot, u64 &ndist, bool &timeout) {
    const int lane = lane_id();
    const Dev &d = a.d;
    const u32 mp = d.mp;
    const float *qrow = a.q + (size_t)qi * mp;
    const u64 *seed_row = a.seed + (size_t)qi * a.L;
    for (u32 i = lane * 4; i < mp; i += 128)
        *reinterpret_cast<float4 *>(s.qv + i) = *reinterpret_cast<const float4 *>(qrow + i);
    seen_clear(a, s);
    __syncwarp();
    float4 qr[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const u32 i = 4u * ((lane & 7) + 8 * t);
        qr[t] = i < mp ? *reinterpret_cast<const float4 *>(s.qv + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (P == 1 && a.tc) {
        // the query as bf16 pairs, and its squared norm over the bf16 values
        float sq = 0.0f;
        u32 *qb = tc_qb(s);
        for (u32 i = lane; 2 * i < d.mb; i += 32) {
            const float x0 = 2 * i < mp ? s.qv[2 * i] : 0.0f, x1 = 2 * i + 1 < mp ? s.qv[2 * i + 1] : 0.0f;
            const u32 w = pack_bf16(x0, x1);
            qb[i] = w;
            const float b0 = __uint_as_float(w << 16), b1 = __uint_as_float(w & 0xFFFF0000u);
            sq = __fmaf_rn(b0, b0, sq);
            sq = __fmaf_rn(b1, b1, sq);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) sq = __fadd_rn(sq, __shfl_xor_sync(FULL, sq, o));
        if (lane == 0) *tc_nq(s) = sq;
        __syncwarp();
    }
    // initial beam: the L nearest members of the entry set E, computed by
    // seed_kernel; the reference words are sampled here
    const u64 *sk = seed_row;
    if (P == 1 && a.tc) {
        // the seeds' keys on the tensor cores, whichever kernel chose them,
        // so that they are the keys this search gives any id; sorted in the stage
        const int bs = min((int)a.stage_rows, 32);   // s.cid holds 32 ids
        for (int b0 = 0; b0 < n0; b0 += bs) {
            const int nb = min(bs, n0 - b0);
            if (lane < nb) s.cid[lane] = key_id(seed_row[b0 + lane]);
            __syncwarp();
            stage_ids<P>(a, s, s.cid, nb, phase, timeout);
            tc_keys(a, s, nb, s.cid, s.bkey + b0);
        }
        u64 *rk = reinterpret_cast<u64 *>(s.stage);
        int np2 = 32;
        while (np2 < n0) np2 <<= 1;
        for (int i = lane; i < np2; i += 32) rk[i] = i < n0 ? s.bkey[i] : KEY_INF;
        __syncwarp();
        warp_sort_u64(rk, np2);
        sk = rk;
    } else if (P != 0 && a.rekey) {
        // seeds ranked by the canonical fp32 distance: every key in the beam
        // must be this precision's distance of its id (an id evaluated again
        // then collapses with its seed), so the seeds are re-keyed and sorted.
        // Their rows go through the stage like a neighbour batch; the keys
        // wait in the beam until the stage is free for the sort.
        const int bs = min((int)a.stage_rows, 32);   // s.cid holds 32 ids
        const int grp = lane >> 3, g = lane & 7;
        const unsigned char *stage = reinterpret_cast<const unsigned char *>(s.stage);
        for (int b0 = 0; b0 < n0; b0 += bs) {
            const int nb = min(bs, n0 - b0);
            if (lane < nb) s.cid[lane] = key_id(seed_row[b0 + lane]);
            __syncwarp();
            stage_ids<P>(a, s, s.cid, nb, phase, timeout);
            for (int r0 = 0; r0 < nb; r0 += 4) {
                const int c = r0 + grp;
                const int cc = c < nb ? c : nb - 1;
                const u32 id = s.cid[cc];
                const float dist = qdist<P>(s.qv, stage + (size_t)cc * a.srow, P == 2 ? d.x8s[id] : 1.0f, (int)mp,
                                            (int)d.metric, g);
                if (c < nb && g == 0) s.bkey[b0 + c] = mkkey(dist, id);
            }
            __syncwarp();
        }
        u64 *rk = reinterpret_cast<u64 *>(s.stage);
        int np2 = 32;
        while (np2 < n0) np2 <<= 1;
        for (int i = lane; i < np2; i += 32) rk[i] = i < n0 ? s.bkey[i] : KEY_INF;
        __syncwarp();
        warp_sort_u64(rk, np2);
        sk = rk;
    }
    for (int i = lane; i < n0; i += 32) {
        const u64 k = sk[i];
        const u32 id = key_id(k);
        s.bkey[i] = k;
        s.bref[i] = ld_ref(d, id);
        s.bflag[i] = 0;
        seen_put(a, s, id);
    }
    int n = n0;
    __syncwarp();
    u32 hops = 0, nexp = 0;
    u32 qcnt = 0;
    u32 *qlog = LOG ? a.elog + (size_t)qi * a.elog_cap : nullptr;
    // slab entries of the predicted next expansion, loaded ahead of use
    u32 pf_id = NIL, pf0 = NIL, pf1 = NIL;
    int lo = 0;   // every beam entry before lo is expanded
    for (;;) {
        int first = -1;
        for (int i0 = lo; i0 < n; i0 += 32) {
            int i = i0 + lane;
            u32 m = __ballot_sync(FULL, i < n && !s.bflag[i]);
            if (m) { first = i0 + __ffs(m) - 1; break; }
        }
        if (first < 0 || hops >= a.max_hops) break;
        hops++;
        lo = first + 1;
        const u64 r = s.bref[first];
        const u64 bkey = s.bkey[first];
        const u32 fid = key_id(bkey);
        const u32 sl = ref_slab(r), deg = sl == NIL ? 0 : ref_deg(r);
        u32 e0 = NIL, e1 = NIL;
        if (fid == pf_id) {
            e0 = pf0; e1 = pf1;
        } else {
            if ((u32)lane < deg) e0 = d.slab[(size_t)sl * d.R + lane].x;
            if ((u32)lane + 32 < deg) e1 = d.slab[(size_t)sl * d.R + lane + 32].x;
        }
        // predict the next expansion: the next unexpanded beam entry
        pf_id = NIL;
        for (int i0 = first + 1; i0 < n; i0 += 32) {
            int i = i0 + lane;
            u32 m = __ballot_sync(FULL, i < n && !s.bflag[i]);
            if (m) {
                const int nx = i0 + __ffs(m) - 1;
                const u64 r2 = s.bref[nx];
                const u32 s2 = ref_slab(r2), d2 = s2 == NIL ? 0 : ref_deg(r2);
                pf_id = key_id(s.bkey[nx]);
                pf0 = (u32)lane < d2 ? d.slab[(size_t)s2 * d.R + lane].x : NIL;
                pf1 = (u32)lane + 32 < d2 ? d.slab[(size_t)s2 * d.R + lane + 32].x : NIL;
                break;
            }
        }
        __syncwarp();
        if (lane == 0) s.bflag[first] = 1;
        if (a.mode == 1 && lane == 0 && !ref_del(r)) a.exp_keys[(size_t)qi * a.max_hops + nexp] = bkey;
        if (!ref_del(r)) nexp++;
        __syncwarp();
        for (u32 j0 = 0; j0 < deg; j0 += 32) {
            u32 nb = j0 == 0 ? e0 : e1;
            if (nb != NIL && seen_has(a, s, nb)) nb = NIL;
            n = eval_merge<P, LOG>(a, s, nb, n, phase, ndist, timeout, lo, qr, qlog, qcnt);
        }
    }
    nexp_tot += hops;
    if (LOG && lane == 0) a.elog_n[qi] = qcnt;
    if (a.mode == 0 && P != 0 && !a.exact) {
        // exact fp32 rerank of the best min(rerank * k, L) live candidates
        u64 *rk = reinterpret_cast<u64 *>(s.stage);
        const int want = (int)min(a.rerank * a.k, a.L);
        int rn = 64;
        while (rn < want) rn <<= 1;
        int c = 0;
        for (int i0 = 0; i0 < n && c < want; i0 += 32) {
            const int i = i0 + lane;
            const bool ok = i < n && !ref_del(s.bref[i]);
            const u32 m = __ballot_sync(FULL, ok);
            const int pos = c + __popc(m & lanemask_lt());
            if (ok && pos < want) rk[pos] = s.bkey[i];
            c = min(want, c + __popc(m));
        }
        __syncwarp();
        const int grp = lane >> 3, g = lane & 7;
        // the fp32 rows go through the stage behind the keys, as many per bulk
        // copy as fit; a stage too small for one row reads them in place
        const u32 rowf = mp * 4u, rkb = (u32)rn * 8u;
        const u32 stb = a.stage_rows * a.srow;
        const int per = stb > rkb ? (int)min(32u, (stb - rkb) / rowf) : 0;
        if (per > 0) {
            unsigned char *rows = reinterpret_cast<unsigned char *>(s.stage) + rkb;
            for (int b0 = 0; b0 < c; b0 += per) {
                const int nb = min(per, c - b0);
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect_tx(s.bar, (u32)nb * rowf);
                }
                __syncwarp();
                if (lane < nb) bulk_g2s(rows + (size_t)lane * rowf, d.x + (size_t)key_id(rk[b0 + lane]) * mp, rowf, s.bar);
                if (!mbar_wait(s.bar, phase, WAIT_LIMIT)) {
                    timeout = true;
                    mbar_wait(s.bar, phase, WAIT_LIMIT);   // let copies in flight land
                }
                phase ^= 1u;
                __syncwarp();
                for (int r0 = 0; r0 < nb; r0 += 4) {
                    const int cc = min(r0 + grp, nb - 1);
                    const u32 id = key_id(rk[b0 + cc]);
                    const float dist = canon_dist<8>(s.qv, reinterpret_cast<const float *>(rows + (size_t)cc * rowf),
                                                     (int)mp, (int)d.metric, g);
                    __syncwarp();
                    if (r0 + grp < nb && g == 0) rk[b0 + cc] = mkkey(dist, id);
                    __syncwarp();
                }
            }
        } else {
            for (int i = lane; i < c; i += 32) bulk_prefetch_l2(d.x + (size_t)key_id(rk[i]) * mp, rowf);
            for (int r0 = 0; r0 < c; r0 += 4) {
                const int cc = min(r0 + grp, c - 1);
                const u32 id = key_id(rk[cc]);
                const float dist = canon_dist<8>(s.qv, d.x + (size_t)id * mp, (int)mp, (int)d.metric, g);
                __syncwarp();
                if (r0 + grp < c && g == 0) rk[cc] = mkkey(dist, id);
                __syncwarp();
            }
        }
        for (int i = c + lane; i < rn; i += 32) rk[i] = KEY_INF;
        __syncwarp();
        warp_sort_u64(rk, rn);
        // equal keys (an id seen twice) are adjacent after the sort: keep one
        u32 outc = 0;
        for (int i0 = 0; i0 < rn; i0 += 32) {
            const int i = i0 + lane;
            const bool ok = rk[i] != KEY_INF && (i == 0 || rk[i] != rk[i - 1]);
            const u32 m = __ballot_sync(FULL, ok);
            const u32 pos = outc + __popc(m & lanemask_lt());
            if (ok && pos < a.k) {
                a.out_ids[(size_t)qi * a.k + pos] = key_id(rk[i]);
                a.out_dist[(size_t)qi * a.k + pos] = key_rho(rk[i]);
            }
            outc += __popc(m);
        }
        for (u32 p = outc + lane; p < a.k; p += 32) {
            a.out_ids[(size_t)qi * a.k + p] = NIL;
            a.out_dist[(size_t)qi * a.k + p] = __int_as_float(0x7f800000);
        }
    } else if (a.mode == 0) {
        // first k beam entries whose sampled delta is 0
        u32 c = 0;
        for (int i0 = 0; i0 < n && c < a.k; i0 += 32) {
            int i = i0 + lane;
            bool ok = i < n && !ref_del(s.bref[i]);
            u32 m = __ballot_sync(FULL, ok);
            u32 pos = c + __popc(m & lanemask_lt());
            if (ok && pos < a.k) {
                a.out_ids[(size_t)qi * a.k + pos] = key_id(s.bkey[i]);
                a.out_dist[(size_t)qi * a.k + pos] = key_rho(s.bkey[i]);
            }
            c += __popc(m);
        }
        for (u32 p = c + lane; p < a.k; p += 32) {
            a.out_ids[(size_t)qi * a.k + p] = NIL;
            a.out_dist[(size_t)qi * a.k + p] = __int_as_float(0x7f800000);
        }
    } else if (lane == 0) {
        a.exp_count[qi] = nexp;
    }
}

// WPB warps (queries in flight) per block; about 24 resident warps per SM.
template <int P, bool LOG = false, int WPB = 4>
__global__ void __launch_bounds__(32 * WPB, 24 / WPB) search_kernel(SearchArgs a) {
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const u32 mp = d.mp;
    const size_t sb = seen_bytes(a);
    const u32 qbytes = a.tc ? d.mb * 2 : 0u;
    const size_t wb = search_warp_bytes(mp, a.L, a.stage_rows, sb, a.srow, qbytes);
    WarpSmem s = carve(smem + warp * wb, mp, a.L, a.stage_rows, sb, a.srow, qbytes);
    if (lane == 0) mbar_init(s.bar, 1);
    __syncwarp();
    u32 phase = 0;
    u64 nexp_tot = 0, ndist = 0;
    bool timeout = false;
    const u32 nq = a.nq_dev ? min(*a.nq_dev, a.nq) : a.nq;
    const int n0 = (int)min(a.L, d.nent_dev ? *d.nent_dev : d.n_entries);
    for (;;) {
        u32 qi = 0;
        if (lane == 0) qi = (u32)atomicAdd(&d.ctr[a.wq], 1ull);
        qi = __shfl_sync(FULL, qi, 0);
        if (qi >= nq) break;
        search_one<P, LOG>(a, s, qi, n0, phase, nexp_tot, ndist, timeout);
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(&d.ctr[C_EXPAND], nexp_tot);
        atomicAdd(&d.ctr[C_DIST], ndist);
        if (timeout) atomicOr(&d.ctr[a.err], (u64)ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------------------------
// Serving ring: a bounded persistent launch that drains a ring of query
// slots in host-mapped memory.  The host writes a query row into its slot,
// then publishes the count of tickets submitted (tail, a release store).  A
// warp claims the next ticket (head, device memory, by compare-and-swap
// while head < tail), seeds the query from the entry set itself, runs the
// BeamSearch and writes the k results into the slot's host-mapped result
// rows, then publishes done[slot] = ticket + 1.  Queries submitted while the
// launch runs are taken as warps free up.  A warp stops claiming once the
// launch has run max_ns nanoseconds (globaltimer) or the ring is closed, so
// every launch ends; slabs are recycled only between launches (Lemma 1).
// ---------------------------------------------------------------------------
struct RingArgs {
    u64 *head;                 // device: tickets claimed
    u64 *dtail;                // device: the submitted count as last read from the host
    u64 *poll_ns;              // device: when a warp last read the host's count
    u64 *dclosed;              // device: the host's stop flag, as last read (zeroed per launch)
    u64 *stats;                // device: queries served, ns seeding, ns searching (accumulated)
    const u64 *tail;           // host-mapped: tickets submitted (host release store)
    const u64 *closed;         // host-mapped: nonzero stops the claims
    u64 *done;                 // host-mapped: done[slot] = ticket + 1 once written
    u32 *served_by;            // host-mapped: launch sequence number that served the slot
    u32 slots, seq;
    u64 max_ns;
};

__device__ __forceinline__ u64 globaltimer_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ u64 ld_acquire_sys(const u64 *p) {
    u64 v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(u64 *p, u64 v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr u32 RING_POLL_LIMIT = 1u << 22;   // each poll sleeps at most RING_SLEEP_MAX ns
constexpr u32 RING_SLEEP_MAX = 8192;        // an idle warp's back-off doubles up to this
constexpr u64 RING_HOST_POLL_NS = 2000;     // the host's count is read about this often

// The L nearest entry points of the query in slot qi, by the same distances
// and merge as seed_kernel (so the seeds equal a batch search's), into
// a.seed + qi * L.  Uses s.qv (the query row), s.bkey and s.nkey.
// One lane's whole distance (the canonical tree of qdist_g with G = 1): the
// row is read in batches of sixteen independent 16-byte loads, so that a batch
// is in flight at once instead of one load per partial.  Partial j still
// accumulates its elements in ascending order and the tree is the same.
template <int P>
__device__ __forceinline__ float lane_dist(const float *__restrict__ q, const void *row, float scale, int mp,
                                           int metric) {
    float p[32];
#pragma unroll
    for (int j = 0; j < 32; j++) p[j] = 0.0f;
    for (int base = 0; base < mp; base += 128) {
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += 16) {
            float4 v[16];
#pragma unroll
            for (int u = 0; u < 16; u++) {
                const int i = base + 4 * (j0 + u);
                v[u] = i < mp ? load4<P>(row, i, scale) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 16; u++) {
                const int i = base + 4 * (j0 + u);
                if (i < mp) {
                    const float4 w = *reinterpret_cast<const float4 *>(q + i);
                    float acc = p[j0 + u];
                    if (metric == 0) {
                        const float d0 = __fsub_rn(w.x, v[u].x), d1 = __fsub_rn(w.y, v[u].y);
                        const float d2 = __fsub_rn(w.z, v[u].z), d3 = __fsub_rn(w.w, v[u].w);
                        acc = __fmaf_rn(d0, d0, acc);
                        acc = __fmaf_rn(d1, d1, acc);
                        acc = __fmaf_rn(d2, d2, acc);
                        acc = __fmaf_rn(d3, d3, acc);
                    } else {
                        acc = __fmaf_rn(w.x, v[u].x, acc);
                        acc = __fmaf_rn(w.y, v[u].y, acc);
                        acc = __fmaf_rn(w.z, v[u].z, acc);
                        acc = __fmaf_rn(w.w, v[u].w, acc);
                    }
                    p[j0 + u] = acc;
                }
            }
        }
    }
#pragma unroll
    for (int hh = 16; hh >= 1; hh >>= 1)
#pragma unroll
        for (int t = 0; t < hh; t++) p[t] = __fadd_rn(p[t], p[t + hh]);
    return metric == 0 ? p[0] : __fsub_rn(1.0f, p[0]);
}

template <int P>
__device__ void ring_seed(const SearchArgs &a, WarpSmem &s, u32 qi) {
    const int lane = lane_id();
    const Dev &d = a.d;
    const u32 mp = d.mp, L = a.L;
    const float *qrow = a.q + (size_t)qi * mp;
    for (u32 i = lane * 4; i < mp; i += 128)
        *reinterpret_cast<float4 *>(s.qv + i) = *reinterpret_cast<const float4 *>(qrow + i);
    __syncwarp();
    // one entry per lane: all 32 rows of a step in flight at once (a warp
    // seeds alone here, with no block-wide tile to stage them in)
    const u32 S = d.nent_dev ? *d.nent_dev : d.n_entries;
    int n = 0;
    u32 e_next = lane < S ? d.entries[lane] : 0u;
    for (u32 t0 = 0; t0 < S; t0 += 32) {
        const u32 e = e_next;
        const bool ok = t0 + lane < S;
        if (t0 + 32 + lane < S) e_next = d.entries[t0 + 32 + lane];
        u64 key = KEY_INF;
        if (ok) key = mkkey(lane_dist<P>(s.qv, row_src<P>(d, e), P == 2 ? d.x8s[e] : 1.0f, (int)mp, (int)d.metric), e);
        n = seed_merge(s.bkey, s.nkey, key, n, (int)L);
    }
    u64 *seed_row = const_cast<u64 *>(a.seed) + (size_t)qi * L;   // the ring's own seed buffer
    for (u32 i = lane; i < L; i += 32) seed_row[i] = (int)i < n ? s.bkey[i] : KEY_INF;
    __syncwarp();
}

template <int P>
__global__ void __launch_bounds__(128, 3) ring_search_kernel(SearchArgs a, RingArgs r) {
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const Dev &d = a.d;
    const size_t sb = seen_bytes(a);
    const u32 qbytes = a.tc ? d.mb * 2 : 0u;
    const size_t wb = search_warp_bytes(d.mp, a.L, a.stage_rows, sb, a.srow, qbytes);
    WarpSmem s = carve(smem + warp * wb, d.mp, a.L, a.stage_rows, sb, a.srow, qbytes);
    if (lane == 0) mbar_init(s.bar, 1);
    __syncwarp();
    u32 phase = 0;
    u64 nexp_tot = 0, ndist = 0, served = 0, seed_ns = 0, search_ns = 0;
    bool timeout = false;
    const u64 t_end = globaltimer_ns() + r.max_ns;
    for (;;) {
        u64 t = KEY_INF;
        if (lane == 0) {
            // Idle warps poll the device copy of the submitted count; one
            // warp at a time, about every RING_HOST_POLL_NS, reads the host's
            // count (acquire) and raises the copy after a fence, so the
            // claiming warp's fence orders its row reads after the host's
            // writes.  Polling the host from every idle warp would flood the
            // link and the SMs' L1 with system-scope acquires.
            u32 nap = 256;
            for (u32 it = 0; it < RING_POLL_LIMIT; it++) {
                // the lifetime bounds the launch even under steady arrivals
                const u64 now = globaltimer_ns();
                if (now >= t_end) break;
                if (*reinterpret_cast<volatile u64 *>(r.dclosed)) break;
                const u64 h = *reinterpret_cast<volatile u64 *>(r.head);
                if (h < *reinterpret_cast<volatile u64 *>(r.dtail)) {
                    if (atomicCAS(r.head, h, h + 1) == h) { t = h; break; }
                    continue;
                }
                const u64 last = *reinterpret_cast<volatile u64 *>(r.poll_ns);
                if (now - last >= RING_HOST_POLL_NS && atomicCAS(r.poll_ns, last, now) == last) {
                    if (ld_acquire_sys(r.closed)) {
                        *reinterpret_cast<volatile u64 *>(r.dclosed) = 1;
                        break;
                    }
                    const u64 tail = ld_acquire_sys(r.tail);
                    __threadfence();
                    atomicMax(reinterpret_cast<unsigned long long *>(r.dtail), (unsigned long long)tail);
                    if (h < tail) continue;
                }
                __nanosleep(nap);
                nap = min(2 * nap, RING_SLEEP_MAX);
            }
        }
        t = __shfl_sync(FULL, t, 0);
        if (t == KEY_INF) break;
        __threadfence_system();   // every lane reads the row after the claim's acquire
        const u32 slot = (u32)(t % r.slots);
        const u64 t0 = globaltimer_ns();
        ring_seed<P>(a, s, slot);
        const u64 t1 = globaltimer_ns();
        const int n0 = (int)min(a.L, d.nent_dev ? *d.nent_dev : d.n_entries);
        search_one<P, false>(a, s, slot, n0, phase, nexp_tot, ndist, timeout);
        __syncwarp();
        if (lane == 0) {
            served++;
            seed_ns += t1 - t0;
            search_ns += globaltimer_ns() - t1;
            r.served_by[slot] = r.seq;
            __threadfence_system();   // the results and served_by before done
            st_release_sys(r.done + slot, t + 1);
        }
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(&d.ctr[C_EXPAND], nexp_tot);
        atomicAdd(&d.ctr[C_DIST], ndist);
        if (served) {
            atomicAdd(r.stats, served);
            atomicAdd(r.stats + 1, seed_ns);
            atomicAdd(r.stats + 2, search_ns);
        }
        if (timeout) atomicOr(&d.ctr[a.err], (u64)ERR_TIMEOUT);
    }
}

// A BF16 search (not the exact-copy form of an fp32 search) takes its keys from
// the tensor cores when the index keeps the copy's norms and the row length
// is a multiple of 32; its stage rows are then padded to an odd number of
// 16-byte chunks, so that ldmatrix's eight row reads fall in distinct banks.
static void set_tc(SearchArgs &a, const Dev &d, u32 prec, bool exact_rows, u32 keys_tc) {
    a.tc = keys_tc && prec == 1 && !exact_rows && d.xbn != nullptr && d.mb % 32 == 0 ? 1u : 0u;
    a.srow = a.tc && (a.rowb / 16) % 2 == 0 ? a.rowb + 16 : a.rowb;
    // a BF16 row is half an fp32 row: as many rows per gather as the fp32
    // shape's stage bytes hold (up to 32), so an expansion needs fewer round
    // trips (measured on the 768-d inner-product index: 497k -> 527k
    // queries/s; FP8 rows at four times the count lost occupancy instead)
    if (prec == 1 && !exact_rows)
        a.stage_rows = std::min<u32>(32, std::max<u32>(a.stage_rows, a.stage_rows * d.mp * 4 / a.srow));
}

// The largest dynamic shared memory a block may opt in to on this device.
static size_t smem_optin_bytes() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    return (size_t)v;
}

// The stage must hold the keys a search sorts there: the rerank candidates
// (rerank * k, at most the beam) and re-keyed seeds (the beam), each rounded
// up to a power of two.
// Returns the fewest stage rows that hold them.
static u32 fit_stage(SearchArgs &a, u32 L, u32 k, u32 rerank, u32 prec, u32 mode) {
    size_t need = 0;
    if (prec != 0 && mode == 0) {
        size_t rn = 64;
        while (rn < std::min<size_t>((size_t)rerank * k, L)) rn <<= 1;
        need = rn;
    }
    if (a.rekey || a.tc) {
        size_t rn = 32;
        while (rn < L) rn <<= 1;
        need = std::max(need, rn);
    }
    const u32 min_rows = std::max<u32>(1, (u32)((need * 8 + a.srow - 1) / a.srow));
    if (a.stage_rows < min_rows) a.stage_rows = min_rows;
    return min_rows;
}

static SeenLayout set_seen(SearchArgs &a, const Dev &d, u32 bits) {
    const SeenLayout l = seen_layout(d.capacity, bits);
    a.seen_bits = bits;
    a.seen_slots = 1u << bits;
    a.seen_tag = l.tag;
    a.seen_shift = l.shift;
    a.seen_tmask = l.tmask;
    a.seen_hmask = l.hmask;
    a.seen_words = l.words;
    return l;
}

cudaError_t launch_ring_search(const Dev &d, float *rows, u32 slots, u32 L, u32 max_hops, u32 k, u32 *out_ids,
                               float *out_dist, u64 *seed, const SearchTuning &tune, u32 blocks, cudaStream_t st,
                               u32 prec, u32 rerank, u64 *head, const u64 *tail, const u64 *closed, u64 *done,
                               u32 *served_by, u32 seq, u64 max_ns) {
    if ((prec == 1 && !d.xb) || (prec == 2 && !d.x8) || prec > 2 || blocks == 0) return cudaErrorInvalidValue;
    SearchArgs a{};
    a.d = d; a.q = rows; a.seed = seed; a.nq_dev = nullptr; a.nq = slots; a.L = L; a.max_hops = max_hops;
    a.mode = 0; a.k = k; a.out_ids = out_ids; a.out_dist = out_dist;
    a.stage_rows = tune.stage_rows;
    const SeenLayout sl = set_seen(a, d, tune.seen_bits);
    a.rowb = prec == 1 ? d.mb * 2 : prec == 2 ? d.m8 : d.mp * 4;
    a.rerank = rerank;
    a.exact = 0;
    a.wq = C_WORK2;
    a.err = C_ERR_S;
    set_tc(a, d, prec, false, tune.keys_tc);
    const u32 min_rows = fit_stage(a, L, k, rerank, prec, 0);
    // head: claimed, device count, last host poll, stop flag, then the statistics
    RingArgs r{head, head + 1, head + 2, head + 3, head + 4, tail, closed, done, served_by, slots, seq, max_ns};
    using K = void (*)(SearchArgs, RingArgs);
    K fn = prec == 1 ? ring_search_kernel<1> : prec == 2 ? ring_search_kernel<2> : ring_search_kernel<0>;
    size_t smem = 4 * search_warp_bytes(d.mp, L, a.stage_rows, sl.bytes, a.srow, a.tc ? d.mb * 2 : 0u);
    while (smem > smem_optin_bytes() && a.stage_rows > min_rows) {
        a.stage_rows--;
        smem = 4 * search_warp_bytes(d.mp, L, a.stage_rows, sl.bytes, a.srow, a.tc ? d.mb * 2 : 0u);
    }
    cudaError_t e = smem_at_least((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, 128, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    e = cudaMemsetAsync(r.dclosed, 0, sizeof(u64), st);   // the stop flag of the launch before
    if (e != cudaSuccess) return e;
    fn<<<blocks, 128, smem, st>>>(a, r);
    return cudaGetLastError();
}

size_t search_smem_bytes(u32 mp, u32 L, u32 stage_rows, u32 seen_bits, u64 capacity, u32 wpb) {
    return (size_t)wpb * search_warp_bytes(mp, L, stage_rows, seen_layout(capacity, seen_bits).bytes, mp * 4);
}

cudaError_t launch_seed(const Dev &d, const float *q, u32 nq, u32 L, u64 *seed, cudaStream_t st, u32 prec,
                        const u32 *nq_dev, const u32 *qsel) {
    if (nq == 0 || (d.n_entries == 0 && !d.nent_dev)) return cudaSuccess;
    if ((prec == 1 && !d.xb) || (prec == 2 && !d.x8) || prec > 2) return cudaErrorInvalidValue;
    const u32 rowb = prec == 1 ? d.mb * 2 : prec == 2 ? d.m8 : d.mp * 4;
    SeedArgs a{d, q, nq_dev, nq, L, seed, rowb, qsel};
    const void *fn = prec == 1 ? (const void *)seed_kernel<1> : prec == 2 ? (const void *)seed_kernel<2>
                                                                          : (const void *)seed_kernel<0>;
    size_t smem = align_up((size_t)SEED_TILE * rowb, 16) + 8 * seed_warp_bytes(d.mp, L);
    cudaError_t e = smem_at_least((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (nq + 7) / 8;
    if (prec == 1) seed_kernel<1><<<blocks, 256, smem, st>>>(a);
    else if (prec == 2) seed_kernel<2><<<blocks, 256, smem, st>>>(a);
    else seed_kernel<0><<<blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_search(const Dev &d, const float *q, u32 nq, u32 L, u32 max_hops, u32 mode, u32 k,
                          u32 *out_ids, float *out_dist, u64 *exp_keys, u32 *exp_count, u64 *seed,
                          const SearchTuning &tune, int num_sms, cudaStream_t st, u32 prec, u32 rerank,
                          const u32 *nq_dev, bool exact_rows, u32 *elog, u32 *elog_n, u32 elog_cap, bool rekey) {
    if (nq == 0) return cudaSuccess;
    if (exact_rows) prec = 1;
    if ((prec == 1 && !d.xb) || (prec == 2 && !d.x8) || prec > 2) return cudaErrorInvalidValue;
    SearchArgs a;
    a.d = d; a.q = q; a.seed = seed; a.nq_dev = nq_dev; a.nq = nq; a.L = L; a.max_hops = max_hops; a.mode = mode;
    a.k = k;
    a.out_ids = out_ids; a.out_dist = out_dist; a.exp_keys = exp_keys; a.exp_count = exp_count;
    a.stage_rows = tune.stage_rows;
    const SeenLayout sl = set_seen(a, d, tune.seen_bits);
    a.rowb = prec == 1 ? d.mb * 2 : prec == 2 ? d.m8 : d.mp * 4;
    a.rerank = rerank;
    a.exact = exact_rows ? 1u : 0u;
    a.rekey = rekey && prec != 0 ? 1u : 0u;
    set_tc(a, d, prec, exact_rows, tune.keys_tc);
    a.wq = mode == 0 ? C_WORK2 : C_WORK;
    a.err = mode == 0 ? C_ERR_S : C_ERR;
    a.elog = elog;
    a.elog_n = elog_n;
    a.elog_cap = elog_cap;
    const bool log = elog != nullptr;
    const u32 wpb = log ? 4u : tune.warps_per_block;
    if (wpb != 2 && wpb != 4 && wpb != 8) return cudaErrorInvalidValue;
    const u32 min_rows = fit_stage(a, L, k, rerank, prec, mode);
    using K = void (*)(SearchArgs);
    K fn = nullptr;
    if (log) fn = prec == 1 ? search_kernel<1, true> : prec == 2 ? search_kernel<2, true> : search_kernel<0, true>;
    else if (wpb == 2) fn = prec == 1 ? search_kernel<1, false, 2> : prec == 2 ? search_kernel<2, false, 2> : search_kernel<0, false, 2>;
    else if (wpb == 8) fn = prec == 1 ? search_kernel<1, false, 8> : prec == 2 ? search_kernel<2, false, 8> : search_kernel<0, false, 8>;
    else fn = prec == 1 ? search_kernel<1> : prec == 2 ? search_kernel<2> : search_kernel<0>;
    size_t smem = (size_t)wpb * search_warp_bytes(d.mp, L, a.stage_rows, sl.bytes, a.srow, a.tc ? d.mb * 2 : 0u);
    // a widened stage (or the bf16 query) that does not fit beside this
    // shape: fewer rows, down to what the sorted keys need
    while (smem > smem_optin_bytes() && a.stage_rows > min_rows) {
        a.stage_rows--;
        smem = (size_t)wpb * search_warp_bytes(d.mp, L, a.stage_rows, sl.bytes, a.srow, a.tc ? d.mb * 2 : 0u);
    }
    cudaError_t e = smem_at_least((const void *)fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, 32 * wpb, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    u32 blocks = (u32)(per_sm * num_sms);
    u32 need = (nq + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(d.ctr + a.wq, 0, sizeof(u64), st);
    if (e != cudaSuccess) return e;
    fn<<<blocks, 32 * wpb, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Evaluation count (diagnostic): for each query, the number of distinct ids
// its BeamSearch evaluated during expansions, not counting the ids of its
// initial beam (the seeds).  That is the size of the exact visited set of
// the search minus the seeds: the evaluations the method itself makes,
// whatever the kernel's lossy cache re-evaluates.  One block per query sorts
// the query's log (bitonic, in shared memory) and the seed ids, then counts.
// ---------------------------------------------------------------------------
__device__ void block_bitonic_u32(u32 *v, u32 n) {   // n a power of two
    for (u32 k = 2; k <= n; k <<= 1)
        for (u32 j = k >> 1; j > 0; j >>= 1) {
            for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
                const u32 l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const u32 x = v[i], y = v[l];
                    if ((x > y) == up) { v[i] = y; v[l] = x; }
                }
            }
            __syncthreads();
        }
}

__global__ void __launch_bounds__(512) eval_unique_kernel(const u32 *elog, const u32 *elog_n, u32 cap,
                                                          const u64 *seed, u32 L, u32 n0, u64 *out) {
    extern __shared__ u32 eu[];
    const u32 qi = blockIdx.x;
    const u32 cnt = elog_n[qi], n = min(cnt, cap);
    u32 np = 1;
    while (np < n) np <<= 1;
    u32 ns = 1;
    while (ns < n0) ns <<= 1;
    u32 *v = eu, *sd = eu + np;
    for (u32 i = threadIdx.x; i < np; i += blockDim.x) v[i] = i < n ? elog[(size_t)qi * cap + i] : NIL;
    for (u32 i = threadIdx.x; i < ns; i += blockDim.x) sd[i] = i < n0 ? key_id(seed[(size_t)qi * L + i]) : NIL;
    __syncthreads();
    block_bitonic_u32(v, np);
    block_bitonic_u32(sd, ns);
    u32 uniq = 0;
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
        const u32 id = v[i];
        if (id == NIL || (i > 0 && v[i - 1] == id)) continue;
        u32 lo = 0, hi = ns;   // is id a seed?
        while (lo < hi) {
            const u32 mid = (lo + hi) >> 1;
            if (sd[mid] < id) lo = mid + 1; else hi = mid;
        }
        uniq += !(lo < ns && sd[lo] == id);
    }
    for (int o = 16; o >= 1; o >>= 1) uniq += __shfl_xor_sync(FULL, uniq, o);
    if ((threadIdx.x & 31) == 0 && uniq) atomicAdd(&out[1], (u64)uniq);
    if (threadIdx.x == 0) {
        atomicAdd(&out[0], (u64)cnt);
        if (cnt > cap) atomicAdd(&out[2], 1ull);   // log overflow (cannot happen when cap = max_hops * R)
    }
}

size_t eval_unique_smem(u32 cap, u32 L) {
    u32 np = 1, ns = 1;
    while (np < cap) np <<= 1;
    while (ns < L) ns <<= 1;
    return (size_t)(np + ns) * 4;
}

cudaError_t launch_eval_unique(const u32 *elog, const u32 *elog_n, u32 cap, const u64 *seed, u32 L, u32 n0, u32 nq,
                               u64 *out, cudaStream_t st) {
    if (nq == 0) return cudaSuccess;
    const size_t smem = eval_unique_smem(cap, L);
    cudaError_t e = smem_at_least((const void *)eval_unique_kernel, smem);
    if (e != cudaSuccess) return e;
    eval_unique_kernel<<<nq, 512, smem, st>>>(elog, elog_n, cap, seed, L, n0, out);
    return cudaGetLastError();
}

}  // namespace etale
