// Exact k nearest live nodes with a tensor-core candidate pass.
//
// Recall@10 (Sec. 5.2) needs the exact top-k over the live set; for the
// 1M x 128 churn workload that is a 10k x 1M x 128 dense contraction per
// round.  The contraction runs on the 5th-generation tensor cores:
//
//   1. gt_prep_rows / gt_prep_queries write bf16 copies of the live rows and
//      the queries (x = hi + lo + e with hi, lo bf16; rows as [hi | lo | hi],
//      queries as [hi | hi | lo], each segment padded to 64) and the norms an
//      error bound needs.  When every lo is zero (data exactly
//      representable in bf16, e.g. integers up to 256) only the first
//      segment is used, otherwise all three (hi.hi + hi.lo + lo.hi).
//   2. gt_tc_kernel: persistent CTAs; TMA (cp.async.bulk.tensor, 128-byte
//      swizzle) streams 256-row boxes of the row copy through a shared
//      memory ring while the query tile stays resident (or, when the query
//      tile's K does not fit shared memory, travels through the ring beside
//      each row box, one 64-column block at a time); one thread issues
//      tcgen05.mma (M = 128, N = 256, bf16 -> fp32) into a double-buffered TMEM
//      accumulator; eight epilogue warps read it with tcgen05.ld and write,
//      per query and per block of 32 rows, the smallest approximate key
//      key = |x|^2 - 2 q.x (L2) or -q.x (IP); dead rows have key +inf.
//   3. gt_rerank_kernel (a warp per query): tau = the 32nd smallest block
//      minimum (or the 2k-th for k > 16); every row of every block whose
//      minimum is <= tau is reranked with the canonical fp32 distance (the
//      same definition the rest of the index uses) into the top k.  Rows
//      left out have approximate keys > tau; an a-priori bound E on
//      |approximate - canonical| certifies that none of them can beat the
//      k-th reranked distance.  Queries that fail the certificate (or have
//      more than 256 candidate blocks) are recomputed by the CUDA-core exact
//      kernel, so the result is always the exact top-k with canonical
//      distances, ties by smaller id.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace etale {
namespace {

constexpr int TC_ROWS = 128;                      // MMA M: queries per query sub-tile
constexpr int TC_ACC = 256;                       // TMEM columns per accumulator buffer
constexpr int TC_KBOX = 64;                       // bf16 per 128-byte swizzle row
constexpr u32 TC_BOX = TC_ROWS * TC_KBOX * 2;     // 16 KB per 128-row TMA box
// Tile shapes: one query sub-tile (M = 128) against 256 rows, or two
// (M = 2 x 128) against 128 rows; both fill a 256-column accumulator.  The
// first reads 96 B of operands from shared memory per MMA cycle instead of
// 128 B (the SM's shared-memory bandwidth), the second half as many rows
// from L2 per query.  On the 1M x 128 workload (10k queries) the first ran
// the candidate pass in 3.5 ms, the second in 4.1 ms, so the plan takes the
// first; the kernel keeps both.
constexpr int TC_MAX_STAGES = 12;
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = (2 + TC_EPI_WARPS) * 32;
constexpr u32 ORD_INF = 0xFF800000u;              // f2ord(+inf)
// kind::f16 instruction descriptor: fp32 accumulator (bits 4-5 = 1), A and B
// bf16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24
__host__ __device__ constexpr u32 tc_idesc(u32 n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((u32)(TC_ROWS >> 4) << 24);
}

struct TcArgs {
    u32 nq, n_tiles, kblocks, n_msub, bn, m_tiles, chunks, tiles_per_chunk, stages;
    u32 all_keys;         // 0: smallest key per block of 32 rows; 1: every key
    u32 stream_a;         // 1: the query boxes travel through the ring (selects gt_tc_kernel<true>)
    const u32 *nq_dev;    // when set, the batch size is read here (nq is its cap); later query tiles are skipped
    u32 ld;               // row length of the output (blocks or keys)
    float s;              // -2 (L2) or -1 (IP)
    const float *xn;      // n_tiles * bn key bases (+inf for dead rows and padding)
    float *out;           // nq x ld
    u32 *err;
};

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(u64 *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, u64 *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle
// layout: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte
// offset), descriptor version 1 (bit 46), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ u64 sw128_desc(u32 saddr) {
    return (u64)((saddr & 0x3FFFFu) >> 4) | ((u64)1 << 16) | ((u64)(1024 >> 4) << 32) | ((u64)1 << 46) |
           ((u64)2 << 61);
}
__device__ __forceinline__ void tc_mma(u32 d, u64 a, u64 b, u32 idesc, u32 acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(u64 *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
// 64 consecutive TMEM columns of this warp's 32 lanes; completes at tmem_wait().
__device__ __forceinline__ void tmem_ld64(u32 taddr, u32 *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- candidate pass ---------------------------------------------------------
// STREAM_A: the query boxes travel through the ring with the row boxes (a
// compile-time choice, so the resident form's MMA issue loop carries no test).
template <bool STREAM_A>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gt_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a) {
    extern __shared__ unsigned char tc_raw[];
    __shared__ __align__(8) u64 full[TC_MAX_STAGES], empty[TC_MAX_STAGES];
    __shared__ __align__(8) u64 a_full, a_empty, t_full[2], t_empty[2], drain;
    __shared__ __align__(16) float xs[2][TC_ACC];    // key bases of the tile in TMEM buffer b
    __shared__ u32 tmem_base;
    __shared__ volatile int abort_flag;
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const u32 items = a.m_tiles * a.chunks;
    const u32 bbox = a.bn * TC_KBOX * 2;            // bytes of one row box
    // query tiles past the batch size in device memory are skipped, the same
    // items by every role
    const u32 nq_eff = a.nq_dev ? min(*a.nq_dev, a.nq) : a.nq;
    const u32 mt_eff = (nq_eff + a.n_msub * TC_ROWS - 1) / (a.n_msub * TC_ROWS);
    // resident: sA holds the query tile (n_msub x kblocks boxes), then the
    // ring of row boxes; streamed: each ring stage is a row box followed by
    // the n_msub query boxes of the same 64 columns
    const u32 abox = a.n_msub * TC_BOX;
    const u32 sbytes = bbox + (STREAM_A ? abox : 0u);
    unsigned char *sA = sm;
    unsigned char *sB = sm + (STREAM_A ? 0u : (size_t)a.kblocks * abox);

    if (threadIdx.x == 0) {
        for (u32 i = 0; i < a.stages; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&a_full, 1);
        mbar_init(&a_empty, 1);
        for (int b = 0; b < 2; b++) {
            mbar_init(&t_full[b], 2);   // the MMA commit + the key-base copy
            mbar_init(&t_empty[b], TC_EPI_WARPS);
        }
        mbar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(2 * TC_ACC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const u32 tmem = tmem_base;

    auto fail = [&]() {
        abort_flag = 1;
        atomicOr(a.err, ERR_TIMEOUT);
    };

    if (warp == 0) {
        // ---- producer: one thread issues every TMA load ----
        if (lane == 0) {
            u32 stage = 0, ph = 0, issued = 0, lastpar = 0, a_issued = 0, a_ph = 0;
            bool first = true;
            for (u32 it = blockIdx.x; it < items && !abort_flag; it += gridDim.x) {
                const u32 mt = it % a.m_tiles, ch = it / a.m_tiles;
                const u32 t0 = ch * a.tiles_per_chunk, t1 = min(a.n_tiles, t0 + a.tiles_per_chunk);
                if (mt >= mt_eff) continue;
                if (!STREAM_A) {
                    if (!first) {
                        if (!mbar_wait(&a_empty, a_ph, WAIT_LIMIT)) { fail(); break; }
                        a_ph ^= 1;
                    }
                    first = false;
                    mbar_expect_tx(&a_full, a.kblocks * abox);
                    for (u32 s = 0; s < a.n_msub; s++)
                        for (u32 kb = 0; kb < a.kblocks; kb++)
                            tma_load_2d(sA + (size_t)(s * a.kblocks + kb) * TC_BOX, &tmA, (int)(kb * TC_KBOX),
                                        (int)((mt * a.n_msub + s) * TC_ROWS), &a_full);
                    a_issued++;
                }
                for (u32 t = t0; t < t1 && !abort_flag; t++) {
                    for (u32 kb = 0; kb < a.kblocks; kb++) {
                        if (!mbar_wait(&empty[stage], ph ^ 1, WAIT_LIMIT)) { fail(); break; }
                        unsigned char *sb = sB + (size_t)stage * sbytes;
                        mbar_expect_tx(&full[stage], sbytes);
                        tma_load_2d(sb, &tmB, (int)(kb * TC_KBOX), (int)(t * a.bn), &full[stage]);
                        if (STREAM_A)
                            for (u32 s = 0; s < a.n_msub; s++)
                                tma_load_2d(sb + bbox + (size_t)s * TC_BOX, &tmA, (int)(kb * TC_KBOX),
                                            (int)((mt * a.n_msub + s) * TC_ROWS), &full[stage]);
                        issued |= 1u << stage;
                        lastpar = (lastpar & ~(1u << stage)) | (ph << stage);
                        if (++stage == a.stages) {
                            stage = 0;
                            ph ^= 1;
                        }
                    }
                }
            }
            // every copy this thread issued has landed before the CTA exits
            for (u32 i = 0; i < a.stages; i++)
                if (issued >> i & 1) mbar_wait(&full[i], lastpar >> i & 1, WAIT_LIMIT);
            if (a_issued) mbar_wait(&a_full, (a_issued - 1) & 1, WAIT_LIMIT);
        }
    } else if (warp == 1) {
        // ---- MMA issuer: one thread ----
        if (lane == 0) {
            u32 stage = 0, ph = 0, a_ph = 0, tcount = 0;
            for (u32 it = blockIdx.x; it < items && !abort_flag; it += gridDim.x) {
                const u32 ch = it / a.m_tiles;
                const u32 t0 = ch * a.tiles_per_chunk, t1 = min(a.n_tiles, t0 + a.tiles_per_chunk);
                if (it % a.m_tiles >= mt_eff) continue;
                if (!STREAM_A) {
                    if (!mbar_wait(&a_full, a_ph, WAIT_LIMIT)) { fail(); break; }
                    a_ph ^= 1;
                    tc_fence_after();
                }
                for (u32 t = t0; t < t1 && !abort_flag; t++, tcount++) {
                    const u32 b = tcount & 1;
                    if (!mbar_wait(&t_empty[b], ((tcount >> 1) & 1) ^ 1, WAIT_LIMIT)) { fail(); break; }
                    tc_fence_after();
                    // the tile's key bases travel with the accumulator: same barrier
                    mbar_expect_tx(&t_full[b], a.bn * 4);
                    bulk_g2s(xs[b], a.xn + (size_t)t * a.bn, a.bn * 4, &t_full[b]);
                    bool ok = true;
                    for (u32 kb = 0; kb < a.kblocks; kb++) {
                        if (!mbar_wait(&full[stage], ph, WAIT_LIMIT)) { ok = false; break; }
                        tc_fence_after();
                        const u32 bb = smem_addr(sB + (size_t)stage * sbytes);
                        const u32 idesc = tc_idesc(a.bn);
#pragma unroll
                        for (u32 k = 0; k < TC_KBOX / 16; k++) {
                            const u64 bd = sw128_desc(bb + k * 32);
                            for (u32 s = 0; s < a.n_msub; s++) {
                                const u32 aa = (STREAM_A ? bb + bbox + s * TC_BOX
                                                           : smem_addr(sA + (size_t)(s * a.kblocks + kb) * TC_BOX)) +
                                               k * 32;
                                tc_mma(tmem + b * TC_ACC + s * TC_ROWS, sw128_desc(aa), bd, idesc, (kb | k) != 0);
                            }
                        }
                        tc_commit(&empty[stage]);
                        if (++stage == a.stages) {
                            stage = 0;
                            ph ^= 1;
                        }
                    }
                    tc_commit(&t_full[b]);
                    if (!ok) {
                        tcount++;   // this tile's key-base copy is in flight too
                        fail();
                        break;
                    }
                }
                if (!STREAM_A) tc_commit(&a_empty);
            }
            // all MMAs and key-base copies issued by this thread are complete
            // before TMEM and shared memory are released
            tc_commit(&drain);
            mbar_wait(&drain, 0, WAIT_LIMIT);
            for (u32 b = 0; b < 2 && b < tcount; b++) {
                const u32 uses = (tcount - b + 1) / 2;     // tiles that used buffer b
                mbar_wait(&t_full[b], (uses - 1) & 1, WAIT_LIMIT);
            }
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31; lane = one query ----
        // group g of four warps: query sub-tile g (two sub-tiles) or row half g (one)
        const int ew = warp - 2, grp = ew >> 2, quarter = warp & 3;
        const int ms = a.n_msub == 2 ? grp : 0, half = a.n_msub == 2 ? 0 : grp;
        {
            const int row = quarter * 32 + lane;
            u32 tcount = 0;
            bool ok = true;
            for (u32 it = blockIdx.x; it < items && ok; it += gridDim.x) {
                const u32 mt = it % a.m_tiles, ch = it / a.m_tiles;
                const u32 t0 = ch * a.tiles_per_chunk, t1 = min(a.n_tiles, t0 + a.tiles_per_chunk);
                if (mt >= mt_eff) continue;
                const u32 q = (mt * a.n_msub + ms) * TC_ROWS + row;
                const bool valid = q < nq_eff;
                float4 *dst = reinterpret_cast<float4 *>(a.out + (size_t)(valid ? q : 0) * a.ld);
                for (u32 t = t0; t < t1; t++, tcount++) {
                    const u32 b = tcount & 1;
                    // every lane waits; the warp goes on together (tcgen05.ld is .sync.aligned)
                    const bool got = !abort_flag && mbar_wait(&t_full[b], (tcount >> 1) & 1, WAIT_LIMIT);
                    if (!__all_sync(FULL, got)) { ok = false; break; }
                    tc_fence_after();
                    const u32 tbase = tmem + ((u32)(quarter * 32) << 16) + b * TC_ACC + grp * TC_ROWS;
                    float bm[TC_ROWS / 32];
                    if (a.all_keys) {
                        u32 r[TC_ROWS];
                        tmem_ld64(tbase, r);
                        tmem_ld64(tbase + 64, r + 64);
                        tmem_wait();
                        const float4 *x4 = reinterpret_cast<const float4 *>(xs[b] + half * TC_ROWS);
                        float4 *o4 = dst + (size_t)(t * a.bn + half * TC_ROWS) / 4;
#pragma unroll
                        for (int j4 = 0; j4 < TC_ROWS / 4; j4++) {
                            const float4 v = x4[j4];
                            const u32 *rr = r + 4 * j4;
                            const float4 kv = make_float4(fmaf(a.s, __uint_as_float(rr[0]), v.x),
                                                          fmaf(a.s, __uint_as_float(rr[1]), v.y),
                                                          fmaf(a.s, __uint_as_float(rr[2]), v.z),
                                                          fmaf(a.s, __uint_as_float(rr[3]), v.w));
                            if (valid) o4[j4] = kv;
                        }
                        // TMEM and the key bases of buffer b are refilled after this
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&t_empty[b]);
                        continue;
                    }
                    {
                        u32 r[TC_ROWS];
                        tmem_ld64(tbase, r);
                        tmem_ld64(tbase + 64, r + 64);
                        tmem_wait();
                        const float4 *x4 = reinterpret_cast<const float4 *>(xs[b] + half * TC_ROWS);
#pragma unroll
                        for (int c = 0; c < TC_ROWS / 32; c++) {
                            float m0 = __int_as_float(0x7f800000), m1 = m0;
#pragma unroll
                            for (int j4 = 0; j4 < 8; j4++) {
                                const float4 v = x4[c * 8 + j4];
                                const u32 *rr = r + c * 32 + 4 * j4;
                                m0 = fminf(m0, fmaf(a.s, __uint_as_float(rr[0]), v.x));
                                m1 = fminf(m1, fmaf(a.s, __uint_as_float(rr[1]), v.y));
                                m0 = fminf(m0, fmaf(a.s, __uint_as_float(rr[2]), v.z));
                                m1 = fminf(m1, fmaf(a.s, __uint_as_float(rr[3]), v.w));
                            }
                            bm[c] = fminf(m0, m1);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&t_empty[b]);
                    if (valid) dst[t * (a.bn / TC_ROWS) + half] = make_float4(bm[0], bm[1], bm[2], bm[3]);
                }
            }
            if (!ok && !abort_flag) fail();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_ACC)
                     : "memory");
    }
}

// ---- bf16 copies and norms ------------------------------------------------
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Four consecutive elements: hi, lo and residual, with the sums an error bound needs.
struct Split4 {
    uint2 hi, lo;
    float sq, lo2, e2;
    bool anylo;
};
__device__ __forceinline__ uint2 pack_bf16x4(float a, float b, float c, float d) {
    const __nv_bfloat162 x = __floats2bfloat162_rn(a, b), y = __floats2bfloat162_rn(c, d);
    return make_uint2(*reinterpret_cast<const u32 *>(&x), *reinterpret_cast<const u32 *>(&y));
}
__device__ __forceinline__ Split4 split4(float4 v) {
    Split4 o;
    const float h0 = bf16_round(v.x), h1 = bf16_round(v.y), h2 = bf16_round(v.z), h3 = bf16_round(v.w);
    const float l0 = bf16_round(v.x - h0), l1 = bf16_round(v.y - h1), l2 = bf16_round(v.z - h2),
                l3 = bf16_round(v.w - h3);
    const float e0 = (v.x - h0) - l0, e1 = (v.y - h1) - l1, e2 = (v.z - h2) - l2, e3 = (v.w - h3) - l3;
    o.hi = pack_bf16x4(h0, h1, h2, h3);
    o.lo = pack_bf16x4(l0, l1, l2, l3);
    o.sq = fmaf(v.w, v.w, fmaf(v.z, v.z, fmaf(v.y, v.y, v.x * v.x)));
    o.lo2 = fmaf(l3, l3, fmaf(l2, l2, fmaf(l1, l1, l0 * l0)));
    o.e2 = fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, e0 * e0)));
    o.anylo = (l0 != 0.0f) | (l1 != 0.0f) | (l2 != 0.0f) | (l3 != 0.0f);
    return o;
}
__device__ __forceinline__ float4 load_row4(const float *r, u32 i, u32 dim, bool on) {
    if (!on || i >= dim) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v = *reinterpret_cast<const float4 *>(r + i);   // rows are padded to a multiple of 4
    if (i + 1 >= dim) v.y = 0.f;
    if (i + 2 >= dim) v.z = 0.f;
    if (i + 3 >= dim) v.w = 0.f;
    return v;
}

// gstat: [0] max |x|^2, [1] max |lo_x|, [2] max |e_x| (fp32 bits), [3] any lo != 0.
// A warp per row, grid-stride; maxima are kept per warp and published once.
// ids (optional): row c is node ids[c]; check_live: rows of deleted or
// never-inserted nodes get key base +inf and a zero copy.
__global__ void gt_prep_rows(Dev d, const u32 *ids, u64 next_id, u32 n_pad, bool check_live, u32 kp1, u32 kb, u32 *B,
                             float *xn, u32 *gstat) {
    const int lane = lane_id();
    const u32 nwarps = (gridDim.x * blockDim.x) >> 5;
    float mx_sq = 0.0f, mx_lo = 0.0f, mx_e = 0.0f;
    bool any_lo = false;
    for (u32 c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_pad; c += nwarps) {
        const u32 id = c < next_id ? (ids ? ids[c] : c) : 0u;
        bool live = c < next_id;
        if (live && check_live) {
            const u64 rf = d.ref[id];
            live = !ref_del(rf) && ref_slab(rf) != NIL;
        }
        float sq = 0.0f, lo2 = 0.0f, e2 = 0.0f;
        bool anylo = false;
        if (c < next_id) {
            const float *xr = d.x + (size_t)id * d.mp;
            uint2 *br = reinterpret_cast<uint2 *>(B + (size_t)c * (kb / 2));
            for (u32 i = 4 * lane; i < kp1; i += 128) {
                const Split4 v = split4(load_row4(xr, i, d.dim, live));
                br[i / 4] = v.hi;
                br[(kp1 + i) / 4] = v.lo;
                br[(2 * kp1 + i) / 4] = v.hi;
                sq += v.sq;
                lo2 += v.lo2;
                e2 += v.e2;
                anylo |= v.anylo;
            }
        }
#pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
            sq += __shfl_xor_sync(FULL, sq, h);
            lo2 += __shfl_xor_sync(FULL, lo2, h);
            e2 += __shfl_xor_sync(FULL, e2, h);
        }
        if (lane == 0) xn[c] = live ? (d.metric == 0 ? sq : 0.0f) : __int_as_float(0x7f800000);
        if (live) {
            mx_sq = fmaxf(mx_sq, sq);
            mx_lo = fmaxf(mx_lo, sqrtf(lo2));
            mx_e = fmaxf(mx_e, sqrtf(e2));
            any_lo |= anylo;
        }
    }
    any_lo = __any_sync(FULL, any_lo);
    if (lane == 0) {
        if (mx_sq > 0.0f) atomicMax(gstat + 0, __float_as_uint(mx_sq));
        if (mx_lo > 0.0f) atomicMax(gstat + 1, __float_as_uint(mx_lo));
        if (mx_e > 0.0f) atomicMax(gstat + 2, __float_as_uint(mx_e));
        if (any_lo) atomicOr(gstat + 3, 1u);
    }
}

// qstat per query: |q|^2, |q|, |lo_q|, |e_q|; copy as [hi | hi | lo]
__global__ void gt_prep_queries(const float *q, u32 mp, u32 dim, u32 nq, u32 kp1, u32 kb, u32 *A, float *qstat,
                                u32 *gstat, const u32 *nq_dev = nullptr) {
    const u32 r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = lane_id();
    if (r >= (nq_dev ? min(*nq_dev, nq) : nq)) return;
    const float *qr = q + (size_t)r * mp;
    uint2 *ar = reinterpret_cast<uint2 *>(A + (size_t)r * (kb / 2));
    float sq = 0.0f, lo2 = 0.0f, e2 = 0.0f;
    bool anylo = false;
    for (u32 i = 4 * lane; i < kp1; i += 128) {
        const Split4 v = split4(load_row4(qr, i, dim, true));
        ar[i / 4] = v.hi;
        ar[(kp1 + i) / 4] = v.hi;
        ar[(2 * kp1 + i) / 4] = v.lo;
        sq += v.sq;
        lo2 += v.lo2;
        e2 += v.e2;
        anylo |= v.anylo;
    }
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        sq += __shfl_xor_sync(FULL, sq, h);
        lo2 += __shfl_xor_sync(FULL, lo2, h);
        e2 += __shfl_xor_sync(FULL, e2, h);
    }
    anylo = __any_sync(FULL, anylo);
    if (lane == 0) {
        qstat[4 * (size_t)r + 0] = sq;
        qstat[4 * (size_t)r + 1] = sqrtf(sq);
        qstat[4 * (size_t)r + 2] = sqrtf(lo2);
        qstat[4 * (size_t)r + 3] = sqrtf(e2);
        if (anylo) atomicOr(gstat + 3, 1u);
    }
}

// ---- the certificate ----------------------------------------------------------
// Lower bound on the canonical fp32 distance of every row whose approximate
// key exceeds LB.  qs: |q|^2, |q|, |lo_q|, |e_q| of the query; gs: max |x|^2,
// max |lo_x|, max |e_x| over the rows (fp32 bits).  K = contracted length.
__device__ double key_lower_bound(int metric, double m, double K, bool split, const float *qs, const u32 *gs,
                                  double LB) {
    const double u = 1.0 / 16777216.0;
    const double qn = qs[0], qa = (double)qs[1] * 1.01, loq = (double)qs[2] * 1.01, eq = (double)qs[3] * 1.01;
    const double X2 = __uint_as_float(gs[0]), X1 = sqrt(X2) * 1.01;
    const double Lx = (double)__uint_as_float(gs[1]) * 1.01, Ex = (double)__uint_as_float(gs[2]) * 1.01;
    // |computed dot - q.x|: the terms the split leaves out, plus fp32 accumulation
    const double dot_res = split ? loq * Lx + (qa + eq) * Ex + eq * (X1 + Ex) : 0.0;
    const double dot_err = dot_res + (K + 2.0) * 2.0 * u * 1.03 * qa * X1;
    if (metric == 0) {
        // norms (fp32 sums of squares), 2 x dot error, rounding of the key
        const double E = 2.0 * ((m + 2.0) * u * qn * 1.01 + (m + 2.0) * u * X2 + 2.0 * dot_err +
                                2.0 * u * (X2 + 2.1 * qa * X1));
        const double y = qn + LB - E;
        // the canonical fp32 distance is within (m + 4) u of the exact one
        return y > 0.0 ? y * (1.0 - 2.0 * (m + 4.0) * u) : -1.0;
    }
    const double E = 2.0 * (dot_err + (m + 2.0) * u * qa * X1 + u * (1.0 + qa * X1));
    return 1.0 + LB - E;
}

// ---- threshold, exact rerank, certificate -------------------------------
constexpr int RR_MAXB = 256;      // candidate blocks a query may keep
constexpr int RR_WARPS = 8;

struct RerankArgs {
    u32 nq, q0, k, nblk, rt, m, kprime, split;
    u64 n_rows;
    const float *q;       // all queries, nq_total x mp fp32
    const float *bmin;    // this group: nq x nblk
    const float *qstat;   // all queries
    const u32 *gstat;
    u32 *out_ids;         // all queries, x k
    float *out_dist;
    u32 *fb;              // queries left to the exact CUDA-core kernel (global indices)
    u32 *fb_count;
    const u32 *err;       // candidate pass error word: nonzero = minima incomplete
};

__global__ void __launch_bounds__(RR_WARPS * 32) gt_rerank_kernel(Dev d, RerankArgs a) {
    __shared__ u32 cblk[RR_WARPS][RR_MAXB];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const u32 li = blockIdx.x * RR_WARPS + warp;
    if (li >= a.nq || *a.err) return;
    const u32 qi = a.q0 + li;
    const float *row = a.bmin + (size_t)li * a.nblk;
    // 1. each lane keeps the four smallest block minima of blocks lane, lane + 32, ...
    u32 t0 = ~0u, t1 = ~0u, t2 = ~0u, t3 = ~0u;
    for (u32 b = lane; b < a.nblk; b += 32) {
        const u32 v = f2ord(__ldg(row + b));
        if (v < t3) {
            if (v < t2) {
                t3 = t2;
                if (v < t1) {
                    t2 = t1;
                    if (v < t0) { t1 = t0; t0 = v; } else t1 = v;
                } else t2 = v;
            } else t3 = v;
        }
    }
    // 2. tau = the rt-th smallest of the 128 kept values (bitwise search on
    //    the order-preserving integer image); at least rt blocks have a
    //    minimum <= tau
    u32 tau = 0;
    for (int bit = 31; bit >= 0; bit--) {
        const u32 tr = tau | (1u << bit);
        const u32 c = (u32)(t0 < tr) + (u32)(t1 < tr) + (u32)(t2 < tr) + (u32)(t3 < tr);
        if (__reduce_add_sync(FULL, c) < a.rt) tau = tr;
    }
    // 3. candidate blocks: minimum <= tau (dead-only blocks have +inf)
    u32 cnt = 0;
    for (u32 b0 = 0; b0 < a.nblk; b0 += 32) {
        const u32 b = b0 + lane;
        const u32 v = b < a.nblk ? f2ord(__ldg(row + b)) : ~0u;
        const bool c = v <= tau && v < ORD_INF;
        const u32 m = __ballot_sync(FULL, c);
        const u32 pos = cnt + __popc(m & lanemask_lt());
        if (c && pos < RR_MAXB) cblk[warp][pos] = b;
        cnt += __popc(m);
    }
    __syncwarp();
    const bool over = cnt > RR_MAXB;
    // 4. exact rerank of every live row of the candidate blocks
    u64 best = KEY_INF;   // sorted across lanes
    const float *qv = a.q + (size_t)qi * d.mp;
    const int grp = lane >> 3, g = lane & 7;
    for (u32 i = 0; i < (over ? 0u : cnt); i++) {
        const u32 b = cblk[warp][i];
        if (lane == 0 && i + 1 < cnt) {
            // the next candidate block's rows on their way to L2
            const u64 r0 = (u64)cblk[warp][i + 1] * 32u;
            const u64 nr = min((u64)32, a.n_rows - r0);
            bulk_prefetch_l2(d.x + r0 * d.mp, (u32)(nr * d.mp * 4u));
        }
        u64 cand = KEY_INF;
        for (int r0 = 0; r0 < 32; r0 += 4) {
            const u32 id = b * 32 + r0 + grp;
            const bool inr = id < a.n_rows;
            bool live = false;
            if (inr) {
                const u64 rf = d.ref[id];
                live = !ref_del(rf) && ref_slab(rf) != NIL;
            }
            // every lane computes (the distance shuffles over the full warp)
            const float dd = canon_dist_wide<8>(qv, d.x + (size_t)(inr ? id : 0u) * d.mp, (int)d.mp, (int)d.metric, g);
            const u64 kk = live ? mkkey(dd, id) : KEY_INF;
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const u64 v = __shfl_sync(FULL, kk, t * 8);
                if (lane == r0 + t) cand = v;
            }
        }
        cand = warp_sort32(cand);
        const u64 rev = __shfl_sync(FULL, cand, 31 - lane);
        best = warp_sort32(best < rev ? best : rev);
    }
    // 5. certificate: every row left out has an approximate key > tau
    const u64 kth = __shfl_sync(FULL, best, a.k - 1);
    bool cert;
    if (over) {
        cert = false;
    } else if (tau >= ORD_INF) {
        cert = true;                                  // every live row was reranked
    } else if (kth == KEY_INF) {
        cert = false;
    } else {
        const double lb = key_lower_bound((int)d.metric, a.m, a.kprime, a.split != 0, a.qstat + 4 * (size_t)qi,
                                          a.gstat, (double)ord2f(tau));
        cert = (double)key_rho(kth) < lb;
    }
    if (cert) {
        if (lane < (int)a.k) {
            a.out_ids[(size_t)qi * a.k + lane] = best == KEY_INF ? NIL : key_id(best);
            a.out_dist[(size_t)qi * a.k + lane] = best == KEY_INF ? __int_as_float(0x7f800000) : key_rho(best);
        }
    } else if (lane == 0) {
        a.fb[atomicAdd(a.fb_count, 1u)] = qi;
    }
}

// ---- seeding: exact top-L of the entry set ---------------------------------
constexpr int SS_CAP = 512;       // candidates a query may keep
constexpr int SS_WARPS = 4;

struct SeedSelArgs {
    u32 nq, L, S, ld, want, m, kprime;
    const float *q;       // nq x mp fp32
    const float *keys;    // nq x ld approximate keys (entry order)
    const float *qstat;
    const u32 *estat;     // maxima over the entry rows
    u64 *seed;            // nq x L
    u32 *fb;              // queries left to the CUDA-core seed kernel
    u32 *ctr;             // [0] their count, [1] error word of the candidate pass
    const u32 *nq_dev;    // when set, the batch size (nq is its cap)
};

// A warp per query: tau = the want-th smallest approximate key; every entry
// with key <= tau is scored with the canonical distance, the scores are
// sorted, and the first L are the seeds if the certificate shows that no
// entry left out can beat the L-th.
__global__ void __launch_bounds__(SS_WARPS * 32) seed_select_kernel(Dev d, SeedSelArgs a) {
    __shared__ u32 cidx[SS_WARPS][SS_CAP];
    __shared__ u64 ckey[SS_WARPS][SS_CAP];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const u32 qi = blockIdx.x * SS_WARPS + warp;
    if (qi >= (a.nq_dev ? min(*a.nq_dev, a.nq) : a.nq) || a.ctr[1]) return;
    const float *row = a.keys + (size_t)qi * a.ld;
    u32 tau = ~0u;                                   // all entries when S <= want
    if (a.S > a.want) {
        // a threshold from every 8th key (16 per lane), kept when the count
        // of keys at or below it lands in [want, SS_CAP]; else (below) the
        // exact want-th smallest key by a bitwise search over all keys
        u32 smp[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const u32 e = 8u * (lane + 32u * j);
            smp[j] = e < a.S ? f2ord(row[e]) : ~0u;
        }
        const u32 rs = a.want / 8 + 8;
        u32 t0 = 0;
        for (int bit = 31; bit >= 0; bit--) {
            const u32 tr = t0 | (1u << bit);
            u32 c = 0;
#pragma unroll
            for (int j = 0; j < 16; j++) c += (u32)(smp[j] < tr);
            if (__reduce_add_sync(FULL, c) < rs) t0 = tr;
        }
        tau = t0;
    }
    // entries with key <= tau, collected and counted in one pass
    auto collect = [&](u32 t) {
        u32 n = 0;
        for (u32 e0 = 0; e0 < a.S; e0 += 32) {
            const u32 e = e0 + lane;
            const bool c = e < a.S && f2ord(row[e]) <= t;
            const u32 m = __ballot_sync(FULL, c);
            const u32 pos = n + __popc(m & lanemask_lt());
            if (c && pos < SS_CAP) cidx[warp][pos] = e;
            n += __popc(m);
        }
        return n;
    };
    u32 cnt = collect(tau);
    if (a.S > a.want && (tau == ~0u || cnt < a.want || cnt > (u32)SS_CAP)) {
        // the sampled threshold missed: the exact want-th smallest key
        tau = 0;
        for (int bit = 31; bit >= 0; bit--) {
            const u32 tr = tau | (1u << bit);
            u32 c2 = 0;
            for (u32 e = lane; e < a.S; e += 32) c2 += (u32)(f2ord(row[e]) < tr);
            if (__reduce_add_sync(FULL, c2) < a.want) tau = tr;
        }
        __syncwarp();
        cnt = collect(tau);
    }
    __syncwarp();
    bool cert = false;
    if (cnt <= SS_CAP) {
        const float *qv = a.q + (size_t)qi * d.mp;
        const int grp = lane >> 3, g = lane & 7;
        if (d.mp <= 128) {
            // the query's elements in registers; four rows per group in flight
            float4 qr[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int i = 4 * (g + 8 * t);
                qr[t] = i < (int)d.mp ? *reinterpret_cast<const float4 *>(qv + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            for (u32 r0 = 0; r0 < cnt; r0 += 16) {
                u32 id[4];
                float dd[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const u32 i = r0 + grp + 4 * u;
                    id[u] = d.entries[cidx[warp][i < cnt ? i : cnt - 1]];
                }
                float4 v[4][4];
#pragma unroll
                for (int u = 0; u < 4; u++) canon_row_q8(d.x + (size_t)id[u] * d.mp, (int)d.mp, g, v[u]);
#pragma unroll
                for (int u = 0; u < 4; u++) dd[u] = canon_dist_q8v(qr, v[u], (int)d.mp, (int)d.metric, g);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const u32 i = r0 + grp + 4 * u;
                    if (i < cnt && g == 0) ckey[warp][i] = mkkey(dd[u], id[u]);
                }
            }
        } else {
            for (u32 r0 = 0; r0 < cnt; r0 += 4) {
                const u32 i = r0 + grp;
                const u32 id = d.entries[cidx[warp][i < cnt ? i : cnt - 1]];
                const float dd = canon_dist_wide<8>(qv, d.x + (size_t)id * d.mp, (int)d.mp, (int)d.metric, g);
                if (i < cnt && g == 0) ckey[warp][i] = mkkey(dd, id);
            }
        }
        const int np = next_pow2((int)cnt);
        for (int i = (int)cnt + lane; i < np; i += 32) ckey[warp][i] = KEY_INF;
        __syncwarp();
        warp_sort_u64(ckey[warp], np);
        if (tau == ~0u) {
            cert = true;                               // every entry was scored
        } else if (cnt >= a.L) {
            const double lb = key_lower_bound((int)d.metric, a.m, a.kprime, true, a.qstat + 4 * (size_t)qi, a.estat,
                                              (double)ord2f(tau));
            cert = (double)key_rho(ckey[warp][a.L - 1]) < lb;
        }
    }
    if (cert) {
        for (u32 i = lane; i < a.L; i += 32) a.seed[(size_t)qi * a.L + i] = i < cnt ? ckey[warp][i] : KEY_INF;
    } else if (lane == 0) {
        a.fb[atomicAdd(a.ctr, 1u)] = qi;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode_bf16(CUtensorMap *m, const void *base, u64 rows, u32 cols, u32 box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {TC_KBOX, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

GtTcPlan gt_tc_plan(u32 dim, u64 next_id, u32 nq) {
    GtTcPlan p{};
    p.kp1 = (dim + TC_KBOX - 1) / TC_KBOX * TC_KBOX;
    p.kb = 3 * p.kp1;
    p.n_pad = (next_id + TC_ACC - 1) / TC_ACC * TC_ACC;
    p.bytes_B = (size_t)next_id * p.kb * 2;
    p.bytes_A = (size_t)nq * p.kb * 2;
    return p;
}

cudaError_t launch_gt_tc_prep(const Dev &d, u64 next_id, const float *q, u32 nq, const GtTcPlan &p,
                              const GtTcBufs &b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.gstat, 0, 8 * sizeof(u32), st);
    if (e != cudaSuccess) return e;
    if (p.n_pad)
        gt_prep_rows<<<(unsigned)std::min<u64>((p.n_pad * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
            d, nullptr, next_id, (u32)p.n_pad, true, p.kp1, p.kb, reinterpret_cast<u32 *>(b.B), b.xn, b.gstat);
    gt_prep_queries<<<(unsigned)(((size_t)nq * 32 + 255) / 256), 256, 0, st>>>(
        q, d.mp, d.dim, nq, p.kp1, p.kb, reinterpret_cast<u32 *>(b.A), b.qstat, b.gstat);
    return cudaGetLastError();
}

void gt_tc_configure(GtTcPlan &p, u32 nq, bool split) {
    p.kprime = split ? p.kb : p.kp1;
    p.split = split;
    p.kblocks = p.kprime / TC_KBOX;
    const u32 smem_max = 227 * 1024 - 1024 - 4096;   // alignment slack, static shared memory
    p.n_msub = 1;
    p.bn = TC_ACC / p.n_msub;
    const u32 bbox = p.bn * TC_KBOX * 2;
    if (p.n_pad == 0) {
        p.usable = false;
        return;
    }
    // the query tile stays resident when it fits beside two ring stages;
    // otherwise its boxes travel through the ring with the row boxes
    p.stream_a = (u64)p.n_msub * p.kblocks * TC_BOX + 2ull * bbox > smem_max;
    if (p.stream_a) {
        p.stages = std::min<u32>(TC_MAX_STAGES, smem_max / (bbox + p.n_msub * TC_BOX));
        p.smem = p.stages * (bbox + p.n_msub * TC_BOX) + 1024;
    } else {
        p.stages = std::min<u32>(TC_MAX_STAGES, (smem_max - p.n_msub * p.kblocks * TC_BOX) / bbox);
        p.smem = p.n_msub * p.kblocks * TC_BOX + p.stages * bbox + 1024;
    }
    p.n_tiles = (u32)(p.n_pad / p.bn);
    p.nblk = (u32)(p.n_pad / 32);
    // queries per pass: the block-minimum buffer stays under 4 GiB
    const u64 cap = std::max<u64>(256, ((4ull << 30) / ((u64)p.nblk * 4)) / 256 * 256);
    p.qgroup = (u32)std::min<u64>(nq, cap);
    p.bytes_bmin = (size_t)p.qgroup * p.nblk * 4;
    p.usable = true;
}

cudaError_t launch_gt_tc(const Dev &d, u32 q0, u32 nq, const GtTcPlan &p, const GtTcBufs &b, u64 next_id,
                         int num_sms, cudaStream_t st) {
    CUtensorMap ta, tb;
    const void *abase = static_cast<const char *>(b.A) + (size_t)q0 * p.kb * 2;
    if (!encode_bf16(&ta, abase, nq, p.kb, TC_ROWS) || !encode_bf16(&tb, b.B, next_id, p.kb, p.bn))
        return cudaErrorInvalidValue;
    TcArgs a{};
    a.nq = nq;
    a.n_tiles = p.n_tiles;
    a.kblocks = p.kblocks;
    a.n_msub = p.n_msub;
    a.bn = p.bn;
    a.m_tiles = (nq + p.n_msub * TC_ROWS - 1) / (p.n_msub * TC_ROWS);
    // chunks of rows: enough work items to fill every SM, with the fewest
    // idle SMs in the last wave
    u32 best_c = 1;
    double best_score = -1e9;
    const u32 cmax = std::max<u32>(1, std::min<u32>(p.n_tiles, 256));
    for (u32 c = 1; c <= cmax; c++) {
        const u64 items = (u64)a.m_tiles * c;
        const u64 waves = (items + num_sms - 1) / num_sms;
        const double eff = (double)items / (double)(waves * num_sms);
        const double score = eff - (items < (u64)num_sms ? 0.5 : 0.0) - 0.002 * c;
        if (score > best_score) {
            best_score = score;
            best_c = c;
        }
    }
    a.tiles_per_chunk = (p.n_tiles + best_c - 1) / best_c;
    a.chunks = (p.n_tiles + a.tiles_per_chunk - 1) / a.tiles_per_chunk;
    a.stages = p.stages;
    a.stream_a = p.stream_a ? 1u : 0u;
    a.all_keys = 0;
    a.ld = p.nblk;
    a.s = d.metric == 0 ? -2.0f : -1.0f;
    a.xn = b.xn;
    a.out = b.bmin;
    a.err = b.err;
    const void *fn = p.stream_a ? (const void *)gt_tc_kernel<true> : (const void *)gt_tc_kernel<false>;
    cudaError_t e = smem_at_least(fn, p.smem);
    if (e != cudaSuccess) return e;
    const u32 items = a.m_tiles * a.chunks;
    const u32 grid = std::min<u32>(items, (u32)num_sms);
    if (p.stream_a) gt_tc_kernel<true><<<grid, TC_THREADS, p.smem, st>>>(ta, tb, a);
    else gt_tc_kernel<false><<<grid, TC_THREADS, p.smem, st>>>(ta, tb, a);
    return cudaGetLastError();
}

cudaError_t launch_gt_rerank(const Dev &d, const float *q, u32 q0, u32 nq, u32 k, const GtTcPlan &p,
                             const GtTcBufs &b, u64 next_id, u32 *out_ids, float *out_dist, cudaStream_t st) {
    RerankArgs r{};
    r.nq = nq;
    r.q0 = q0;
    r.k = k;
    r.nblk = p.nblk;
    r.rt = k <= 16 ? 32 : 2 * k;
    r.m = d.dim;
    r.kprime = p.kprime;
    r.split = p.split;
    r.n_rows = next_id;
    r.q = q;
    r.bmin = b.bmin;
    r.qstat = b.qstat;
    r.gstat = b.gstat;
    r.out_ids = out_ids;
    r.out_dist = out_dist;
    r.fb = b.fb;
    r.fb_count = b.gstat + 4;
    r.err = b.err;
    gt_rerank_kernel<<<(nq + RR_WARPS - 1) / RR_WARPS, RR_WARPS * 32, 0, st>>>(d, r);
    return cudaGetLastError();
}

// ---- seeding on tensor cores ----------------------------------------------
SeedTcPlan seed_tc_plan(u32 dim, u32 n_entry, u32 nq) {
    SeedTcPlan p{};
    p.kp1 = (dim + TC_KBOX - 1) / TC_KBOX * TC_KBOX;
    p.kb = 3 * p.kp1;
    p.s_pad = (n_entry + TC_ACC - 1) / TC_ACC * TC_ACC;
    const u32 smem_max = 227 * 1024 - 1024 - 4096;
    const u32 bbox = TC_ACC * TC_KBOX * 2;
    const u32 abytes = (p.kb / TC_KBOX) * TC_BOX;
    p.usable = n_entry > 0;
    // the query tile resident when it fits beside two ring stages, else streamed
    p.stream_a = abytes + 2 * bbox > smem_max;
    if (p.stream_a) {
        p.stages = std::min<u32>(TC_MAX_STAGES, smem_max / (bbox + TC_BOX));
        p.smem = p.stages * (bbox + TC_BOX) + 1024;
    } else {
        p.stages = std::min<u32>(TC_MAX_STAGES, (smem_max - abytes) / bbox);
        p.smem = abytes + p.stages * bbox + 1024;
    }
    p.bytes_E = (size_t)n_entry * p.kb * 2;
    p.bytes_A = (size_t)nq * p.kb * 2;
    p.bytes_keys = (size_t)nq * p.s_pad * 4;
    return p;
}

cudaError_t launch_seed_tc_entries(const Dev &d, u32 S, const SeedTcPlan &p, const SeedTcBufs &b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.estat, 0, 8 * sizeof(u32), st);
    if (e != cudaSuccess || p.s_pad == 0) return e;
    gt_prep_rows<<<(unsigned)std::min<u64>(((u64)p.s_pad * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(
        d, d.entries, S, p.s_pad, false, p.kp1, p.kb, reinterpret_cast<u32 *>(b.E), b.en, b.estat);
    return cudaGetLastError();
}

cudaError_t launch_seed_tc(const Dev &d, const float *q, u32 nq, u32 S, u32 L, u64 *seed, const SeedTcPlan &p,
                           const SeedTcBufs &b, int num_sms, cudaStream_t st, const u32 *nq_dev) {
    if (nq == 0 || S == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(b.ctr, 0, 8 * sizeof(u32), st);
    if (e != cudaSuccess) return e;
    gt_prep_queries<<<(unsigned)(((size_t)nq * 32 + 255) / 256), 256, 0, st>>>(
        q, d.mp, d.dim, nq, p.kp1, p.kb, reinterpret_cast<u32 *>(b.A), b.qstat, b.ctr + 4, nq_dev);
    CUtensorMap ta, tb;
    if (!encode_bf16(&ta, b.A, nq, p.kb, TC_ROWS) || !encode_bf16(&tb, b.E, S, p.kb, TC_ACC))
        return cudaErrorInvalidValue;
    TcArgs a{};
    a.nq = nq;
    a.n_tiles = p.s_pad / TC_ACC;
    a.kblocks = p.kb / TC_KBOX;
    a.n_msub = 1;
    a.bn = TC_ACC;
    a.m_tiles = (nq + TC_ROWS - 1) / TC_ROWS;
    u32 best_c = 1;
    double best_score = -1e9;
    for (u32 c = 1; c <= a.n_tiles; c++) {
        const u64 items = (u64)a.m_tiles * c;
        const u64 waves = (items + num_sms - 1) / num_sms;
        const double score = (double)items / (double)(waves * num_sms) - 0.02 * c;
        if (score > best_score) {
            best_score = score;
            best_c = c;
        }
    }
    a.tiles_per_chunk = (a.n_tiles + best_c - 1) / best_c;
    a.chunks = (a.n_tiles + a.tiles_per_chunk - 1) / a.tiles_per_chunk;
    a.stages = p.stages;
    a.stream_a = p.stream_a ? 1u : 0u;
    a.nq_dev = nq_dev;
    a.all_keys = 1;
    a.ld = p.s_pad;
    a.s = d.metric == 0 ? -2.0f : -1.0f;
    a.xn = b.en;
    a.out = b.keys;
    a.err = b.ctr + 1;
    const void *fn = p.stream_a ? (const void *)gt_tc_kernel<true> : (const void *)gt_tc_kernel<false>;
    e = smem_at_least(fn, p.smem);
    if (e != cudaSuccess) return e;
    const u32 items = a.m_tiles * a.chunks;
    if (p.stream_a) gt_tc_kernel<true><<<std::min<u32>(items, (u32)num_sms), TC_THREADS, p.smem, st>>>(ta, tb, a);
    else gt_tc_kernel<false><<<std::min<u32>(items, (u32)num_sms), TC_THREADS, p.smem, st>>>(ta, tb, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SeedSelArgs r{};
    r.nq = nq;
    r.L = L;
    r.S = S;
    r.ld = p.s_pad;
    r.want = L + 32;
    r.m = d.dim;
    r.kprime = p.kb;
    r.q = q;
    r.keys = b.keys;
    r.qstat = b.qstat;
    r.estat = b.estat;
    r.seed = seed;
    r.fb = b.fb;
    r.ctr = b.ctr;
    r.nq_dev = nq_dev;
    seed_select_kernel<<<(nq + SS_WARPS - 1) / SS_WARPS, SS_WARPS * 32, 0, st>>>(d, r);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // queries the certificate did not cover: the exact CUDA-core seed, with
    // the count read on the device
    return launch_seed(d, q, nq, L, seed, st, 0, b.ctr, b.fb);
}

}  // namespace etale
