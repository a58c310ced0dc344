// common.cuh — device-side building blocks of the ETALE index for sm_103a.
//
// State (Definition 1): vectors x[C][mp] fp32 (rows zero-padded to mp, a
// multiple of 4, so every row is 16-byte aligned for bulk copies), one 64-bit
// reference word per id, and a pool of P slabs of R entries {u32 id; f32 rho}.
// Slabs come from a free stack and go back through a retired stack that the
// host recycles between launches (Sec. 3.3, Lemma 1).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace etale {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u32 NIL = 0xFFFFFFFFu;
constexpr u64 KEY_INF = ~0ull;
constexpr u32 FULL = 0xFFFFFFFFu;
constexpr int MAX_R = 64;

// ---- device error word (bit flags, OR-ed by kernels, read by the host) ----
enum : u32 {
    ERR_NOMEM = 1u,        // free stack ran dry during a launch
    ERR_TIMEOUT = 2u,      // a bounded mbarrier wait gave up
    ERR_CAS = 4u,          // a deterministic-mode CAS lost (must not happen)
    ERR_OVERFLOW = 8u,     // a scratch list overflowed its bound
};

// ---- pool / statistics counters (one u64 array in device memory) ----------
enum : int {
    C_FREE = 0,        // entries on the free stack at launch start
    C_POP = 1,         // pops taken during the current launch
    C_RET = 2,         // entries on the retired stack
    C_ERR = 3,         // error bits
    C_PUBLISH = 4,
    C_CAS_RETRY = 5,
    C_DROPPED = 6,
    C_EXPAND = 7,
    C_DIST = 8,
    C_WORK = 9,        // work-queue counter (reset before each persistent launch)
    C_WORK2 = 10,
    C_COUNT_A = 11,    // scratch counts produced on the device
    C_COUNT_B = 12,
    C_ERR_S = 13,      // error bits of query searches (kept apart from writers')
    C_RECYCLED = 14,   // blocks of the recycle launch that have finished copying
    C_INEXACT = 15,    // ingested rows whose bf16 copy differs from the fp32 row
    C_WK = 16,         // work tallies of the writer kernels: two words per WK_* kind
    C_NCTR = 32
};
// Work a writer kernel's method needs, tallied per warp and added once at the
// warp's end: word 0 the bytes of vector rows gathered (distinct rows of each
// prune or distance step, in the copy the step reads), word 1 the bytes of
// graph state read or written (reference words, slab entries, tombstone bits).
// Lists that pass between kernels (candidate keys, offers, replacement sets)
// are not counted.
enum : int { WK_PRUNE = 0, WK_OFFER, WK_REFINE, WK_REPAIR_K, WK_REPAIR_FOLD, WK_COMPACT, WK_N };
static_assert(C_WK + 2 * WK_N <= C_NCTR, "work tallies exceed the counter array");

// ---- reference word r(u) = <delta, d, s>: bit 63 delta, bits 48..55 d,
//      bits 0..31 s (NIL = no slab).  Same packing as the paper's single
//      64-bit word; the bit positions are this library's choice.  Bit 56 (P)
//      is a hint of this library's own: set when the list was written by a
//      RobustPrune (or is such a list with entries removed), so that no entry
//      is dropped by an earlier one; a plain insertion clears it.
__host__ __device__ __forceinline__ u64 ref_pack(u32 del, u32 d, u32 s) {
    return ((u64)(del & 1u) << 63) | ((u64)(d & 0xFFu) << 48) | (u64)s;
}
__host__ __device__ __forceinline__ u32 ref_del(u64 r) { return (u32)(r >> 63); }
__host__ __device__ __forceinline__ u32 ref_deg(u64 r) { return (u32)(r >> 48) & 0xFFu; }
__host__ __device__ __forceinline__ u32 ref_slab(u64 r) { return (u32)r; }
__host__ __device__ __forceinline__ u32 ref_pruned(u64 r) { return (u32)(r >> 56) & 1u; }

// ---- (rho, id) total order: fp32 bits mapped to an unsigned order ---------
__host__ __device__ __forceinline__ u32 fbits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    u32 u;
    __builtin_memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float bitsf(u32 u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    __builtin_memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ u32 f2ord(float f) {
    u32 u = fbits(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ord2f(u32 o) {
    u32 u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    return bitsf(u);
}
__host__ __device__ __forceinline__ u64 mkkey(float rho, u32 id) {
    return ((u64)f2ord(rho) << 32) | id;
}
__host__ __device__ __forceinline__ u32 key_id(u64 k) { return (u32)k; }
__host__ __device__ __forceinline__ float key_rho(u64 k) { return ord2f((u32)(k >> 32)); }

// ---- index view passed by value to every kernel ---------------------------
struct Dev {
    float *x;          // C x mp
    u64 *ref;          // C
    uint2 *slab;       // P x R   {id, rho bits}
    u32 *free_stack;   // P
    u32 *retired;      // P
    u64 *ctr;          // C_NCTR counters
    u32 *entries;      // n_entry
    const u32 *nent_dev;  // current |E| in device memory (read by query kernels,
                          // so a captured graph follows later updates)
    u32 dim, mp, R, metric;
    float alpha2;
    u32 n_entries;
    u64 capacity, pool;
    u32 stage_bytes;   // per-warp RobustPrune row stage (0: rows read from L2)
    u32 gram;          // 1: domination tests of small prunes use the tensor-core Gram tile
    // reduced-precision copies (query search only)
    unsigned short *xb;  // C x mb bf16 bits (nullptr if not kept)
    float *xbn;          // C: |bf16 row|^2, for the tensor-core keys of BF16 searches
    unsigned char *x8;   // C x m8 e4m3 codes (nullptr if not kept)
    float *x8s;          // C per-vector scales
    u32 mb, m8;          // row strides in elements (16-byte rows)
    u32 slab_batch;      // free slabs a warp pops at once (1..32; see WarpSlabs)
    // Round state in device memory (RS_* words), set only for launches recorded
    // into a round graph: kernels then take next_id and the first id of the
    // current insert from here instead of from their arguments, so that one
    // recorded round stays valid as the index grows.  nullptr otherwise.
    u64 *rs;
};

enum : int {
    RS_NEXT = 0,      // ids handed out so far
    RS_FIRST = 1,     // first id of the insert being run
    RS_LIVE = 2,      // live count at the last entry-set recomputation
    RS_DELETED = 3,   // ids tombstoned since the host last read the state
    RS_N = 8
};
// next_id for a kernel whose argument (a grid bound) may exceed it.
__device__ __forceinline__ u64 dev_next_id(const Dev &d, u64 arg) { return d.rs ? min(arg, d.rs[RS_NEXT]) : arg; }
__device__ __forceinline__ u32 dev_first(const Dev &d, u32 arg) { return d.rs ? (u32)d.rs[RS_FIRST] : arg; }

// ---- canonical distance ------------------------------------------------------
// Element i belongs to partial j = (i mod 128) / 4.  Each partial is a fused
// multiply-add chain over its elements in ascending i, from +0.  The 32
// partials are combined as q[j] = p[j] + p[j + h] for h = 16, 8, 4, 2, 1.
// G lanes (an aligned group) cooperate on one distance: lane g of the group
// owns partials g, g + G, g + 2G, ...; the tree levels h >= G are summed in
// the lane, the levels h < G by xor shuffles.  Every lane of the group
// returns the same value.  Explicit _rn intrinsics keep the compiler from
// contracting or reordering anything.
template <int G>
__device__ __forceinline__ float canon_dist(const float *__restrict__ a, const float *__restrict__ b,
                                            int mp, int metric, int g) {
    constexpr int T = 32 / G;
    float p[T];
#pragma unroll
    for (int t = 0; t < T; t++) {
        const int j = g + G * t;
        float acc = 0.0f;
        for (int base = 0; base < mp; base += 128) {
            const int i = base + 4 * j;
            if (i < mp) {
                const float4 u = *reinterpret_cast<const float4 *>(a + i);
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

// canon_dist<G> with the column blocks outermost: the T loads of one block
// are in flight together (more registers, fewer round trips for rows read
// from global memory); every p[t] sums its elements in the same order, so
// the result is bit-identical to canon_dist<G>.
template <int G>
__device__ __forceinline__ float canon_dist_wide(const float *__restrict__ a, const float *__restrict__ b,
                                                 int mp, int metric, int g) {
    constexpr int T = 32 / G;
    float p[T];
#pragma unroll
    for (int t = 0; t < T; t++) p[t] = 0.0f;
    for (int base = 0; base < mp; base += 128) {
        float4 u[T], v[T];
#pragma unroll
        for (int t = 0; t < T; t++) {
            const int i = base + 4 * (g + G * t);
            if (i < mp) {
                u[t] = *reinterpret_cast<const float4 *>(a + i);
                v[t] = *reinterpret_cast<const float4 *>(b + i);
            }
        }
#pragma unroll
        for (int t = 0; t < T; t++) {
            const int i = base + 4 * (g + G * t);
            if (i < mp) {
                float acc = p[t];
                if (metric == 0) {
                    float d0 = __fsub_rn(u[t].x, v[t].x), d1 = __fsub_rn(u[t].y, v[t].y);
                    float d2 = __fsub_rn(u[t].z, v[t].z), d3 = __fsub_rn(u[t].w, v[t].w);
                    acc = __fmaf_rn(d0, d0, acc);
                    acc = __fmaf_rn(d1, d1, acc);
                    acc = __fmaf_rn(d2, d2, acc);
                    acc = __fmaf_rn(d3, d3, acc);
                } else {
                    acc = __fmaf_rn(u[t].x, v[t].x, acc);
                    acc = __fmaf_rn(u[t].y, v[t].y, acc);
                    acc = __fmaf_rn(u[t].z, v[t].z, acc);
                    acc = __fmaf_rn(u[t].w, v[t].w, acc);
                }
                p[t] = acc;
            }
        }
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

// canon_dist<8> for rows of at most 128 floats, in two steps so that several
// rows' loads can be in flight: canon_row_q8 loads this lane's four row float4
// (elements 4 (g + 8 t) .. + 3, t = 0..3; zero past the row), canon_dist_q8v
// reduces them against the query's four float4 held in registers, with the
// same operations in the same order as canon_dist<8>.
__device__ __forceinline__ void canon_row_q8(const float *__restrict__ b, int mp, int g, float4 (&v)[4]) {
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int i = 4 * (g + 8 * t);
        v[t] = i < mp ? *reinterpret_cast<const float4 *>(b + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ float canon_dist_q8v(const float4 (&qr)[4], const float4 (&v)[4], int mp, int metric,
                                                int g) {
    float p[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int i = 4 * (g + 8 * t);
        float acc = 0.0f;
        if (i < mp) {
            const float4 u = qr[t];
            if (metric == 0) {
                float d0 = __fsub_rn(u.x, v[t].x), d1 = __fsub_rn(u.y, v[t].y);
                float d2 = __fsub_rn(u.z, v[t].z), d3 = __fsub_rn(u.w, v[t].w);
                acc = __fmaf_rn(d0, d0, acc);
                acc = __fmaf_rn(d1, d1, acc);
                acc = __fmaf_rn(d2, d2, acc);
                acc = __fmaf_rn(d3, d3, acc);
            } else {
                acc = __fmaf_rn(u.x, v[t].x, acc);
                acc = __fmaf_rn(u.y, v[t].y, acc);
                acc = __fmaf_rn(u.z, v[t].z, acc);
                acc = __fmaf_rn(u.w, v[t].w, acc);
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

// ---- small warp helpers -------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ u32 lanemask_lt() {
    u32 m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Ascending bitonic sort of n (a power of two, >= 32) u64 keys in shared
// memory by one warp.
__device__ __forceinline__ void warp_sort_u64(u64 *a, int n) {
    const int lane = lane_id();
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n; i += 32) {
                int l = i ^ j;
                if (l > i) {
                    u64 x = a[i], y = a[l];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { a[i] = y; a[l] = x; }
                }
            }
            __syncwarp();
        }
    }
}

// Bitonic sort of one u64 per lane across the warp (ascending by lane).
__device__ __forceinline__ u64 warp_sort32(u64 v) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            u64 o = __shfl_xor_sync(FULL, v, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            u64 lo = v < o ? v : o, hi = v < o ? o : v;
            v = (lower == up) ? lo : hi;
        }
    }
    return v;
}

// Four independent warp_sort32 networks interleaved: the same result as four
// calls, with their shuffles in flight together.
__device__ __forceinline__ void warp_sort32x4(u64 (&v)[4]) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const bool take_lo = ((lane & j) == 0) == ((lane & k) == 0);
            u64 o[4];
#pragma unroll
            for (int q = 0; q < 4; q++) o[q] = __shfl_xor_sync(FULL, v[q], j);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const u64 lo = v[q] < o[q] ? v[q] : o[q], hi = v[q] < o[q] ? o[q] : v[q];
                v[q] = take_lo ? lo : hi;
            }
        }
    }
}

__device__ __forceinline__ int next_pow2(int n) {
    int p = 32;
    while (p < n) p <<= 1;
    return p;
}

// ---- slab pool: AllocSlab / RetireSlab (Sec. 3.3) ----------------------------
// Inside one launch the free stack is only popped and the retired stack only
// pushed, each through one atomic counter; the host-ordered recycle kernel
// moves retired entries back between launches.
__device__ __forceinline__ void retire_slab(const Dev &d, u32 s) {
    u64 j = atomicAdd(&d.ctr[C_RET], 1ull);
    d.retired[j] = s;
}

// Per-warp batches of slab pops and retirements (lane j holds entry j of
// each batch).  A warp pops d.slab_batch free slabs with one atomic and pushes
// its retirements 32 at a time; before the kernel ends, ws_finish pushes the
// popped slabs it did not use onto the retired stack, so the recycle step
// between launches (Lemma 1) returns them.  No slab is reused inside the
// launch that retired it, as before.  The host sets slab_batch to 1 when the
// free pool is too small for every resident warp to hold a batch.
struct WarpSlabs {
    u32 pop_slab, ret_slab;
    u32 spare;           // warp-uniform: a slab written for a lost CAS, never linked
    int npop, nret;      // warp-uniform
    u64 npub, nretry;    // counted on every lane, added once
};
__device__ __forceinline__ void ws_init(WarpSlabs &w) {
    w.pop_slab = NIL;
    w.ret_slab = NIL;
    w.spare = NIL;
    w.npop = w.nret = 0;
    w.npub = w.nretry = 0;
}
__device__ __forceinline__ u32 ws_pop(const Dev &d, WarpSlabs &w) {
    const int lane = threadIdx.x & 31;
    if (w.spare != NIL) {   // reuse the slab of a lost CAS: no reader can hold it
        const u32 s = w.spare;
        w.spare = NIL;
        return s;
    }
    if (w.npop == 0) {
        const u32 K = d.slab_batch < 1 ? 1u : (d.slab_batch > 32 ? 32u : d.slab_batch);
        u64 i0 = 0;
        if (lane == 0) i0 = atomicAdd(&d.ctr[C_POP], (u64)K);
        i0 = __shfl_sync(0xffffffffu, i0, 0);
        const u64 nfree = d.ctr[C_FREE];
        const bool ok = (u32)lane < K && i0 + lane < nfree;
        w.pop_slab = ok ? d.free_stack[nfree - 1 - (i0 + lane)] : NIL;
        w.npop = __popc(__ballot_sync(0xffffffffu, ok));
        if (w.npop == 0) {
            if (lane == 0) atomicOr(&d.ctr[C_ERR], (u64)ERR_NOMEM);
            return NIL;
        }
    }
    w.npop--;
    return __shfl_sync(0xffffffffu, w.pop_slab, w.npop);
}
__device__ __forceinline__ void ws_flush(const Dev &d, WarpSlabs &w) {
    const int lane = threadIdx.x & 31;
    if (w.nret == 0) return;
    u64 j0 = 0;
    if (lane == 0) j0 = atomicAdd(&d.ctr[C_RET], (u64)w.nret);
    j0 = __shfl_sync(0xffffffffu, j0, 0);
    if (lane < w.nret) d.retired[j0 + lane] = w.ret_slab;
    w.nret = 0;
}
__device__ __forceinline__ void ws_retire(const Dev &d, WarpSlabs &w, u32 s) {
    if ((threadIdx.x & 31) == (u32)w.nret) w.ret_slab = s;
    if (++w.nret == 32) ws_flush(d, w);
}
__device__ __forceinline__ void ws_finish(const Dev &d, WarpSlabs &w) {
    const int lane = threadIdx.x & 31;
    if (w.spare != NIL) {
        ws_retire(d, w, w.spare);
        w.spare = NIL;
    }
    ws_flush(d, w);
    if (w.npop > 0) {
        u64 j0 = 0;
        if (lane == 0) j0 = atomicAdd(&d.ctr[C_RET], (u64)w.npop);
        j0 = __shfl_sync(0xffffffffu, j0, 0);
        if (lane < w.npop) d.retired[j0 + lane] = w.pop_slab;
        w.npop = 0;
    }
    if (lane == 0) {
        if (w.npub) atomicAdd(&d.ctr[C_PUBLISH], w.npub);
        if (w.nretry) atomicAdd(&d.ctr[C_CAS_RETRY], w.nretry);
    }
}

// Warp-cooperative Publish(u, N) (Algorithm 1).  All 32 lanes call it with
// the same arguments; ids/rho hold the n <= R entries (shared memory) and
// `snap` is the reference word the caller read before building N.  The CAS
// installs <delta of snap, n, fresh slab> only if r(u) still equals snap;
// returns true on success.  On a lost CAS false is returned (the caller
// retries or drops the update) and the fresh slab, which was never linked
// into any reference and so cannot be read by anyone else, is kept as the
// warp's spare: the next publication writes into it instead of popping, so
// retries under contention do not drain the pool.  A spare left at the end of
// a launch is retired.
// pruned: the new list's P bit (see ref_pruned).
__device__ __forceinline__ bool warp_publish(const Dev &d, WarpSlabs &ws, u32 u, const u32 *ids,
                                             const float *rho, int n, u64 snap, bool pruned) {
    const int lane = lane_id();
    const u32 s2 = ws_pop(d, ws);
    if (s2 == NIL) return false;
    uint2 *dst = d.slab + (u64)s2 * d.R;
    for (int j = lane; j < n; j += 32) dst[j] = make_uint2(ids[j], __float_as_uint(rho[j]));
    __threadfence();           // slab contents visible before the reference
    __syncwarp();
    int ok = 0;
    if (lane == 0) {
        const u64 nw = ref_pack(ref_del(snap), (u32)n, s2) | ((u64)(pruned ? 1u : 0u) << 56);   // carry the deletion flag
        ok = atomicCAS(&d.ref[u], snap, nw) == snap;
    }
    ok = __shfl_sync(FULL, ok, 0);
    if (ok) {
        if (ref_slab(snap) != NIL) ws_retire(d, ws, ref_slab(snap));
        ws.npub++;
    } else {
        ws.spare = s2;
        ws.nretry++;
    }
    return ok != 0;
}

__device__ __forceinline__ u64 ld_ref(const Dev &d, u32 id) {
    return *reinterpret_cast<volatile const u64 *>(d.ref + id);
}

// ---- warp-level bf16 tensor-core helpers (mma.sync m16n8k16, fp32 accumulation) ----
__device__ __forceinline__ void ldsm_x4(u32 &r0, u32 &r1, u32 &r2, u32 &r3, u32 addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16_16816(float *c, u32 a0, u32 a1, u32 a2, u32 a3, u32 b0, u32 b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ u32 pack_bf16(float lo, float hi) {
    u32 r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// ---- bulk (TMA, non-tensor) copies into shared memory with an mbarrier -----
__device__ __forceinline__ u32 smem_addr(const void *p) {
    return static_cast<u32>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(u64 *bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64 *bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Fire-and-forget bulk prefetch of [src, src + bytes) into L2 (src 16-byte
// aligned, bytes a multiple of 16); nothing waits on it.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, u32 bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, u32 bytes, u64 *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Bounded wait on the given phase parity.  Returns false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(u64 *bar, u32 parity, u32 limit) {
    for (u32 it = 0; it < limit; it++) {
        u32 done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
constexpr u32 WAIT_LIMIT = 1u << 22;   // each try_wait suspends ~1 us at most

}  // namespace etale
