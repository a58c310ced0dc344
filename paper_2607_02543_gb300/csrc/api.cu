// api.cu — the C ABI (include/etale.h): memory ownership, phase
// orchestration and the host side of the epoch discipline.  Each phase is a
// separate launch on the caller's stream and every phase that publishes is
// followed by the recycle launch (Sec. 3.3, Lemma 1, Definition 2).
#include <algorithm>
#include <atomic>
#include <thread>
#include <chrono>
#include <initializer_list>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/etale.h"
#include "common.cuh"
#include "internal.h"

using namespace etale;

namespace etale {
std::atomic<unsigned long long> g_kernel_launches{0};
}

namespace {

// Message of the last failed call on this thread (any index), so that a
// search thread and a writer thread never share one string.
thread_local std::string t_last_error = "no error";

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int pins = 0;   // round graphs that recorded this buffer's address
};

// A buffer a round graph recorded is never reallocated while the graph lives.
bool grow(DevBuf &b, size_t bytes) {
    if (b.bytes >= bytes) return true;
    if (b.pins) return false;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    b.bytes = want;
    return true;
}

template <class T>
T *as(DevBuf &b) { return reinterpret_cast<T *>(b.p); }

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

u32 bits_for(u64 v) {
    u32 b = 1;
    while (b < 32 && (v >> b) != 0) b++;
    return b;
}

}  // namespace

struct etale_index {
    int device = 0, num_sms = 0, smem_optin = 0;
    int writer_sms = 0;   // SMs the grids of update kernels are sized for (etale_set_writer_share)
    etale_config cfg{};
    u32 dim = 0, mp = 0, R = 0, metric = 0;
    u64 capacity = 0, pool = 0;
    float alpha2 = 0.f;
    // index memory
    float *x = nullptr;
    u64 *ref = nullptr;
    uint2 *slab = nullptr;
    u32 *free_stack = nullptr, *retired = nullptr, *entries = nullptr;
    u64 *ctr = nullptr;
    unsigned short *xb = nullptr;   // bf16 copy
    float *xbn = nullptr;           // squared norms of the bf16 copy's rows
    unsigned char *x8 = nullptr;    // fp8 copy
    float *x8s = nullptr;
    u32 mb = 0, m8 = 0;
    u32 search_prec = 0;
    u32 insert_prec = 0;            // precision of the insert BeamSearch gathers
    bool rows_exact = true;         // every ingested row's bf16 copy is exact (C_INEXACT == 0)
    u32 *nent_dev = nullptr;        // |E| in device memory
    u64 *rs = nullptr;              // round state (RS_* words) of recorded rounds
    int round_graphs = 0;           // live graphs that pin index buffers (round graphs, tensor-seeded query graphs)
    bool graph_pending = false;     // a round graph ran since the host state was read
    cudaEvent_t graph_ev = nullptr; // recorded after the last round-graph launch
    u64 *host_ctr = nullptr;   // pinned mirror
    // scratch
    DevBuf stage, qpad, out_ids, out_dist, exp_keys, exp_count, F_id, F_rho, F_n;
    DevBuf of_key, of_val, of_key2, of_val2, of_src, of_rho, seg_flags, seg_scan, seg_start, sort_scr, scan_scr;
    DevBuf live_flags, live_rank, live_scan_scr, tomb_bits;
    DevBuf del_ids, del_vals, del_ids2, del_vals2, del_ok, del_scan, dt, pair_key, pair_val, pair_key2, pair_val2,
        pair_K, pair_Kn, pair_flags, pair_scan, pair_seg, counts;
    DevBuf ex_del, ex_hs, ex_deg, ex_ids, ex_rho, seed, refine_spill;
    // query-search scratch, separate from the writer's so that one search
    // call and one update call can run at the same time (concurrent mode)
    DevBuf s_stage, s_qpad, s_out_ids, s_out_dist, s_seed;
    // ground truth on tensor cores
    DevBuf gt_A, gt_B, gt_xn, gt_qstat, gt_gstat, gt_fb, gt_bmin;
    u32 gt_path = 0;
    u64 gt_fallbacks = 0;
    // seeding on tensor cores
    DevBuf sd_E, sd_en, sd_estat, sd_A, sd_qstat, sd_keys, sd_fb, sd_ctr;
    bool seed_tc = false;   // configured and the shapes fit
    u64 *host_ctr_s = nullptr;        // pinned, search side
    u64 *host_ctr_st = nullptr;       // pinned, etale_stats
    cudaStream_t stat_stream = nullptr;
    std::mutex mu;                    // guards search_ev and its validity
    cudaEvent_t search_ev = nullptr;  // recorded after every query search
    bool search_ev_valid = false;
    cudaEvent_t search_ev2 = nullptr; // the same for ring launches on a ring's second stream
    bool search_ev2_valid = false;
    bool concurrent = false;
    // host-side state
    u64 next_id = 0, live = 0, tombs = 0, reclaimed = 0;
    std::atomic<u32> n_entries{0};
    u64 free_lb = 0;
    u64 device_bytes = 0;
    SearchTuning tune;

    // phase timing (opt-in)
    static constexpr int MAXREC = 2048;
    bool prof = false;
    std::vector<cudaEvent_t> pev;
    int prec_phase[MAXREC];
    int nrec = 0, open_phase = -1;
    double pms[ETALE_PH_COUNT] = {0};
    u64 pcnt[ETALE_PH_COUNT] = {0};

    SeedTcBufs seed_bufs() const {
        SeedTcBufs b{};
        b.E = sd_E.p;
        b.A = sd_A.p;
        b.en = static_cast<float *>(sd_en.p);
        b.qstat = static_cast<float *>(sd_qstat.p);
        b.keys = static_cast<float *>(sd_keys.p);
        b.estat = static_cast<u32 *>(sd_estat.p);
        b.fb = static_cast<u32 *>(sd_fb.p);
        b.ctr = static_cast<u32 *>(sd_ctr.p);
        return b;
    }
    Dev dev() const {
        Dev d;
        d.x = x; d.ref = ref; d.slab = slab; d.free_stack = free_stack; d.retired = retired; d.ctr = ctr;
        d.entries = entries; d.dim = dim; d.mp = mp; d.R = R; d.metric = metric; d.alpha2 = alpha2;
        d.n_entries = n_entries.load(std::memory_order_relaxed); d.capacity = capacity; d.pool = pool; d.stage_bytes = cfg.stage_kb << 10;
        d.gram = cfg.gram == 2 ? 1u : 0u;
        d.xb = xb; d.xbn = xbn; d.x8 = x8; d.x8s = x8s; d.mb = mb; d.m8 = m8;
        // warps pop 8 free slabs at a time when the free pool covers every
        // resident warp's batch many times over (else one, as Algorithm 1)
        d.slab_batch = free_lb >= (u64)num_sms * 64 * 8 * 2 ? 8u : 1u;
        d.nent_dev = nent_dev;
        d.rs = nullptr;
        return d;
    }

    etale_status fail(etale_status s, const char *fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        t_last_error = buf;
        return s;
    }
    etale_status cuda_fail(cudaError_t e, const char *where) {
        return fail(ETALE_ECUDA, "%s: %s", where, cudaGetErrorString(e));
    }
};

#define CK(expr, where)                                                     \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) return idx->cuda_fail(_e, where);            \
    } while (0)
#define CK2(ix, expr, where)                                                \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) return (ix)->cuda_fail(_e, where);           \
    } while (0)

namespace {

// Fold recorded phase events into the accumulators (the stream has been
// synchronised by the caller).
void prof_flush(etale_index *idx) {
    for (int i = 0; i < idx->nrec; i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, idx->pev[2 * i], idx->pev[2 * i + 1]) == cudaSuccess) {
            idx->pms[idx->prec_phase[i]] += ms;
            idx->pcnt[idx->prec_phase[i]]++;
        }
    }
    cudaGetLastError();
    idx->nrec = 0;
}

void prof_begin(etale_index *idx, int phase, cudaStream_t st) {
    if (!idx->prof) return;
    if (idx->nrec == etale_index::MAXREC) {
        cudaStreamSynchronize(st);
        prof_flush(idx);
    }
    cudaEventRecord(idx->pev[2 * idx->nrec], st);
    idx->open_phase = phase;
}

void prof_end(etale_index *idx, cudaStream_t st) {
    if (!idx->prof || idx->open_phase < 0) return;
    cudaEventRecord(idx->pev[2 * idx->nrec + 1], st);
    idx->prec_phase[idx->nrec++] = idx->open_phase;
    idx->open_phase = -1;
}

struct PhaseScope {
    etale_index *idx;
    cudaStream_t st;
    PhaseScope(etale_index *i, int ph, cudaStream_t s) : idx(i), st(s) { prof_begin(i, ph, s); }
    ~PhaseScope() { prof_end(idx, st); }
};

// Read the device counters (synchronises the stream).
etale_status read_ctr(etale_index *idx, cudaStream_t st) {
    CK(cudaMemcpyAsync(idx->host_ctr, idx->ctr, C_NCTR * sizeof(u64), cudaMemcpyDeviceToHost, st), "read counters");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (idx->prof) prof_flush(idx);
    return ETALE_OK;
}

etale_status check_device_errors(etale_index *idx, cudaStream_t st) {
    etale_status s = read_ctr(idx, st);
    if (s != ETALE_OK) return s;
    idx->free_lb = idx->host_ctr[C_FREE];
    const u64 e = idx->host_ctr[C_ERR];
    if (e) {
        u64 z = 0;
        cudaMemcpy(idx->ctr + C_ERR, &z, sizeof z, cudaMemcpyHostToDevice);
        if (e & ERR_TIMEOUT) return idx->fail(ETALE_ETIMEOUT, "a bounded device wait gave up");
        if (e & ERR_NOMEM) return idx->fail(ETALE_ENOMEM, "slab pool exhausted during a launch");
        if (e & ERR_CAS) return idx->fail(ETALE_EINTERNAL, "a publication lost a CAS that had no competitor");
        if (e & ERR_OVERFLOW) return idx->fail(ETALE_EINTERNAL, "a candidate list overflowed its bound");
        return idx->fail(ETALE_EINTERNAL, "device error bits 0x%llx", e);
    }
    return ETALE_OK;
}

// After round-graph launches the device holds the live count, the deletions
// made and the entry-set size; read them back before a call that uses the
// host's copies (waits for the last launch).
etale_status settle(etale_index *idx) {
    if (!idx->graph_pending) return ETALE_OK;
    CK(cudaEventSynchronize(idx->graph_ev), "wait for the round graph");
    u64 rs[RS_N];
    u32 nent = 0;
    CK(cudaMemcpy(rs, idx->rs, sizeof rs, cudaMemcpyDeviceToHost), "read round state");
    CK(cudaMemcpy(&nent, idx->nent_dev, 4, cudaMemcpyDeviceToHost), "read entry count");
    CK(cudaMemcpy(idx->host_ctr, idx->ctr, C_NCTR * sizeof(u64), cudaMemcpyDeviceToHost), "read counters");
    CK(cudaMemset(idx->rs + RS_DELETED, 0, sizeof(u64)), "reset round state");
    idx->graph_pending = false;
    idx->live = rs[RS_LIVE];
    idx->reclaimed += idx->tombs + rs[RS_DELETED];
    idx->tombs = 0;
    idx->n_entries = nent;
    idx->free_lb = idx->host_ctr[C_FREE];
    const u64 e = idx->host_ctr[C_ERR] | idx->host_ctr[C_ERR_S];
    if (e) {
        CK(cudaMemset(idx->ctr + C_ERR, 0, sizeof(u64)), "clear error");
        CK(cudaMemset(idx->ctr + C_ERR_S, 0, sizeof(u64)), "clear error");
        if (e & ERR_TIMEOUT) return idx->fail(ETALE_ETIMEOUT, "round graph: a bounded device wait gave up");
        if (e & ERR_NOMEM) return idx->fail(ETALE_ENOMEM, "round graph: slab pool exhausted during a launch");
        return idx->fail(ETALE_EINTERNAL, "round graph: device error bits 0x%llx", e);
    }
    return ETALE_OK;
}

// Query-search counterpart of check_device_errors: its own pinned buffer and
// error word, so that it never touches the writer's.
etale_status check_search_errors(etale_index *idx, cudaStream_t st) {
    CK(cudaMemcpyAsync(idx->host_ctr_s, idx->ctr, C_NCTR * sizeof(u64), cudaMemcpyDeviceToHost, st), "read counters");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (idx->prof && !idx->concurrent) prof_flush(idx);
    const u64 e = idx->host_ctr_s[C_ERR_S];
    if (e) {
        CK(cudaMemsetAsync(idx->ctr + C_ERR_S, 0, sizeof(u64), st), "clear error");
        CK(cudaStreamSynchronize(st), "synchronize");
        if (e & ERR_TIMEOUT) return idx->fail(ETALE_ETIMEOUT, "a bounded device wait gave up");
        return idx->fail(ETALE_EINTERNAL, "device error bits 0x%llx", e);
    }
    return ETALE_OK;
}

// Concurrent mode: a writer call first waits (on its stream) for the last
// query search issued so far, then returns the slabs retired by the previous
// writer call to the free stack.  Any search that could still read one of
// those slabs was issued before this call started (Proposition 2's separation
// of searches from slab reuse, enforced with an event instead of a device
// barrier).
etale_status writer_begin(etale_index *idx, cudaStream_t st);

// Make sure a phase that may pop `need` slabs cannot exhaust the pool.
etale_status ensure_pool(etale_index *idx, u64 need, cudaStream_t st) {
    if (idx->free_lb >= need) {
        idx->free_lb -= need;
        return ETALE_OK;
    }
    etale_status s = read_ctr(idx, st);
    if (s != ETALE_OK) return s;
    idx->free_lb = idx->host_ctr[C_FREE];
    if (idx->free_lb < need)
        return idx->fail(ETALE_ENOMEM, "slab pool: %llu free, a phase may need %llu", (unsigned long long)idx->free_lb,
                         (unsigned long long)need);
    idx->free_lb -= need;
    return ETALE_OK;
}

// Lock-free fold chunk: as many slots as the free pool covers at two slabs
// each (one publication plus a retried one), at least one.  In concurrent
// mode nothing is recycled mid-call, so the whole remainder must fit.
etale_status lockfree_chunk(etale_index *idx, u64 remaining, u64 *chunk, cudaStream_t st);

etale_status recycle_now(etale_index *idx, cudaStream_t st) {
    PhaseScope ps(idx, ETALE_PH_RECYCLE, st);
    CK(launch_recycle(idx->dev(), st), "recycle");
    g_kernel_launches++;
    return ETALE_OK;
}

etale_status lockfree_chunk(etale_index *idx, u64 remaining, u64 *chunk, cudaStream_t st) {
    u64 want = remaining * 2;
    if (idx->free_lb < want) {
        etale_status s = read_ctr(idx, st);
        if (s != ETALE_OK) return s;
        idx->free_lb = idx->host_ctr[C_FREE];
    }
    u64 c = std::min<u64>(remaining, idx->free_lb / 2);
    if (idx->concurrent && c < remaining)
        return idx->fail(ETALE_ENOMEM, "slab pool: %llu free, a concurrent-mode update may need %llu",
                         (unsigned long long)idx->free_lb, (unsigned long long)want);
    if (c == 0) return idx->fail(ETALE_ENOMEM, "slab pool exhausted (%llu free)", (unsigned long long)idx->free_lb);
    idx->free_lb -= 2 * c;
    *chunk = c;
    return ETALE_OK;
}

etale_status writer_begin(etale_index *idx, cudaStream_t st) {
    if (!idx->concurrent) return ETALE_OK;
    {
        std::lock_guard<std::mutex> lk(idx->mu);
        if (idx->search_ev_valid) CK(cudaStreamWaitEvent(st, idx->search_ev, 0), "wait for searches");
        if (idx->search_ev2_valid) CK(cudaStreamWaitEvent(st, idx->search_ev2, 0), "wait for searches");
    }
    return recycle_now(idx, st);
}

// The recycle step between launches (Sec. 3.3).  In concurrent mode the
// retired slabs stay retired until the next writer call (writer_begin).
etale_status recycle(etale_index *idx, cudaStream_t st) {
    if (idx->concurrent) return ETALE_OK;
    PhaseScope ps(idx, ETALE_PH_RECYCLE, st);
    CK(launch_recycle(idx->dev(), st), "recycle");
    g_kernel_launches++;
    return ETALE_OK;
}

etale_status recompute_entries(etale_index *idx, cudaStream_t st) {
    const u64 n = idx->next_id;
    const u32 S = (u32)(idx->live < idx->cfg.n_entry ? idx->live : idx->cfg.n_entry);
    idx->n_entries = S;
    // the device copy of |E| (read by query kernels and captured graphs) is
    // written on the writer's stream, in order with the entry-set update
    CK(launch_set_u32(idx->nent_dev, S, st), "entry count");
    if (S == 0 || n == 0) return ETALE_OK;
    if (!grow(idx->live_flags, n * 4) || !grow(idx->live_rank, n * 4) ||
        !grow(idx->live_scan_scr, scan_scratch_elems((u32)n) * 4))
        return idx->fail(ETALE_ENOMEM, "scratch allocation (entries)");
    ScanScratch ss;
    scan_scratch_carve(ss, as<u32>(idx->live_scan_scr), (u32)n);
    Dev d = idx->dev();
    PhaseScope ps(idx, ETALE_PH_ENTRIES, st);
    CK(launch_live_flags(d, n, as<u32>(idx->live_flags), st), "live flags");
    CK(exclusive_scan(as<u32>(idx->live_flags), as<u32>(idx->live_rank), (u32)n, ss, st), "live scan");
    CK(launch_entries_select(d, n, as<u32>(idx->live_flags), as<u32>(idx->live_rank), idx->live, S, st),
       "entries select");
    g_kernel_launches += 3;
    if (idx->seed_tc) {
        const SeedTcPlan p = seed_tc_plan(idx->dim, S, 0);
        if (!grow(idx->sd_E, p.bytes_E) || !grow(idx->sd_en, (size_t)p.s_pad * 4) || !grow(idx->sd_estat, 64))
            return idx->fail(ETALE_ENOMEM, "entry-set copy");
        CK(launch_seed_tc_entries(d, S, p, idx->seed_bufs(), st), "entry-set copy");
        g_kernel_launches++;
    }
    return ETALE_OK;
}

// Sort offers by target (stable), segment them, fold (deterministic) or
// publish each offer (lock-free).
// `targets` bounds the number of distinct targets (each publishes at most
// once per phase in deterministic mode; lock-free retries are rare and a dry
// pool is reported by the device).
etale_status run_offers(etale_index *idx, u32 nslots, u64 targets, cudaStream_t st) {
    Dev d = idx->dev();
    Offers of{as<u32>(idx->of_key), as<u32>(idx->of_val), as<u32>(idx->of_key2), as<u32>(idx->of_val2),
              as<u32>(idx->of_src), as<float>(idx->of_rho), nslots};
    const bool lockfree = idx->cfg.mode == ETALE_MODE_LOCKFREE;
    u64 *seg_count = as<u64>(idx->counts) + 0;
    if (lockfree) {
        // every offer publishes on its own (a lost CAS retires one more slab):
        // cut the slots into chunks the free pool covers, recycling between
        for (u64 lo = 0; lo < nslots;) {
            u64 chunk;
            etale_status s = lockfree_chunk(idx, nslots - lo, &chunk, st);
            if (s != ETALE_OK) return s;
            {
                PhaseScope ps(idx, ETALE_PH_OFFER_FOLD, st);
                CK(launch_offer_fold(d, of, nullptr, seg_count, idx->cfg.cas_budget, idx->writer_sms, st, (u32)lo,
                                     (u32)(lo + chunk)),
                   "offer fold");
            }
            g_kernel_launches++;
            s = recycle(idx, st);
            if (s != ETALE_OK) return s;
            lo += chunk;
        }
        return ETALE_OK;
    }
    etale_status s = ensure_pool(idx, std::min<u64>(nslots, targets), st);
    if (s != ETALE_OK) return s;
    if (!lockfree) {
        PhaseScope ps(idx, ETALE_PH_OFFER_SORT, st);
        SortScratch ss;
        sort_scratch_carve(ss, as<u32>(idx->sort_scr), nslots);
        CK(radix_sort_pairs(of.key, of.val, of.key_alt, of.val_alt, nslots, bits_for(idx->capacity), ss, st),
           "offer sort");
        ScanScratch sc;
        scan_scratch_carve(sc, as<u32>(idx->scan_scr), nslots);
        CK(make_segments(of.key, nslots, (u32)idx->capacity, as<u32>(idx->seg_flags), as<u32>(idx->seg_scan),
                         as<u32>(idx->seg_start), seg_count, sc, st),
           "offer segments");
        g_kernel_launches += 3 * ((bits_for(idx->capacity) + 7) / 8) * 2 + 4;
    }
    {
        PhaseScope ps(idx, ETALE_PH_OFFER_FOLD, st);
        CK(launch_offer_fold(d, of, as<u32>(idx->seg_start), seg_count, lockfree ? idx->cfg.cas_budget : 0,
                             idx->writer_sms, st),
           "offer fold");
    }
    g_kernel_launches++;
    return recycle(idx, st);
}

bool size_delete_scratch(etale_index *idx, u64 n) {
    const u64 R = idx->R, slots = n * R;
    return grow(idx->del_ids, n * 4) && grow(idx->del_vals, n * 4) && grow(idx->del_ids2, n * 4) &&
           grow(idx->del_vals2, n * 4) && grow(idx->del_ok, n * 4) && grow(idx->del_scan, n * 4) &&
           grow(idx->dt, n * 4) && grow(idx->pair_key, slots * 4) && grow(idx->pair_val, slots * 4) &&
           grow(idx->pair_key2, slots * 4) && grow(idx->pair_val2, slots * 4) &&
           grow(idx->pair_K, slots * R * 8) && grow(idx->pair_Kn, slots * 4) &&
           grow(idx->pair_flags, slots * 4) && grow(idx->pair_scan, slots * 4) &&
           grow(idx->pair_seg, (slots + 1) * 4) && grow(idx->counts, 64) &&
           grow(idx->sort_scr, sort_scratch_elems((u32)std::max<u64>(slots, n)) * 4) &&
           grow(idx->scan_scr, scan_scratch_elems((u32)std::max<u64>(slots, n)) * 4);
}

etale_status size_batch_scratch(etale_index *idx, u64 b) {
    const u64 R = idx->R, H = idx->cfg.max_hops ? idx->cfg.max_hops : 4ull * idx->cfg.build_beam;
    const u64 slots = b * R;
    bool ok = grow(idx->exp_keys, b * H * 8) && grow(idx->exp_count, b * 4) && grow(idx->F_id, slots * 4) &&
              grow(idx->F_rho, slots * 4) && grow(idx->F_n, b * 4) && grow(idx->of_key, slots * 4) &&
              grow(idx->of_val, slots * 4) && grow(idx->of_key2, slots * 4) && grow(idx->of_val2, slots * 4) &&
              grow(idx->of_src, slots * 4) && grow(idx->of_rho, slots * 4) && grow(idx->seg_flags, slots * 4) &&
              grow(idx->seg_scan, slots * 4) && grow(idx->seg_start, (slots + 1) * 4) &&
              grow(idx->sort_scr, sort_scratch_elems((u32)slots) * 4) &&
              grow(idx->scan_scr, scan_scratch_elems((u32)slots) * 4) && grow(idx->counts, 64);
    return ok ? ETALE_OK : idx->fail(ETALE_ENOMEM, "scratch allocation (insert batch of %llu)", (unsigned long long)b);
}

// fp32 BeamSearches may gather the bf16 copy: it holds every stored row
// exactly, so the distances are those of the fp32 rows.  Not in concurrent
// mode, where a row ingested during a search could be inexact.
bool exact_rows(const etale_index *idx) {
    return idx->cfg.exact_rows == 1 && idx->rows_exact && idx->xb && !idx->concurrent;
}

// The BeamSearch launch shape with its row stage shrunk until a block's shared
// memory fits the device (long rows); results do not depend on the stage.
SearchTuning fit_tuning(const etale_index *idx, u32 L, SearchTuning t) {
    while (t.stage_rows > 1 &&
           search_smem_bytes(idx->mp, L, t.stage_rows, t.seen_bits, idx->capacity, t.warps_per_block) > (size_t)idx->smem_optin)
        t.stage_rows >>= 1;
    return t;
}

// Seeds of nq BeamSearches (top-L of the entry set): tensor cores with a
// certified exact rerank when they apply, else the CUDA-core kernel; both
// give the same seeds.  The tensor path ranks by the canonical fp32 distance
// also for a reduced-precision search (*fp32_keys = true): that search then
// re-keys its seeds in its own precision (launch_search's rekey).
static etale_status seed_batch(etale_index *idx, const Dev &d, const float *q, u32 nq, u32 L, u64 *seed, u32 prec,
                               cudaStream_t st, int sms = 0, bool *fp32_keys = nullptr) {
    const u32 S = idx->n_entries;
    if (fp32_keys) *fp32_keys = false;
    if ((prec == 0 || fp32_keys) && idx->seed_tc && !idx->concurrent && S > 0 && nq >= 32) {
        const SeedTcPlan p = seed_tc_plan(idx->dim, S, nq);
        if (!grow(idx->sd_A, p.bytes_A) || !grow(idx->sd_qstat, (size_t)nq * 16) ||
            !grow(idx->sd_keys, p.bytes_keys) || !grow(idx->sd_fb, (size_t)nq * 4) || !grow(idx->sd_ctr, 64))
            return idx->fail(ETALE_ENOMEM, "seed staging");
        CK(launch_seed_tc(d, q, nq, S, L, seed, p, idx->seed_bufs(), sms ? sms : idx->num_sms, st), "seed (tensor)");
        g_kernel_launches += 4;
        if (fp32_keys) *fp32_keys = prec != 0;
        return ETALE_OK;
    }
    CK(launch_seed(d, q, nq, L, seed, st, prec), "seed");
    g_kernel_launches++;
    return ETALE_OK;
}

etale_status insert_subbatch(etale_index *idx, u32 first, u32 b, cudaStream_t st) {
    Dev d = idx->dev();
    const u32 L = idx->cfg.build_beam;
    const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * L;
    const u32 R = idx->R;
    const u32 slots = b * R;
    Offers of{as<u32>(idx->of_key), as<u32>(idx->of_val), as<u32>(idx->of_key2), as<u32>(idx->of_val2),
              as<u32>(idx->of_src), as<float>(idx->of_rho), slots};
    // 1. BeamSearch of every member on the graph before the sub-batch
    if (!grow(idx->seed, (size_t)b * L * 8)) return idx->fail(ETALE_ENOMEM, "seed buffer");
    bool rekey = false;
    {
        PhaseScope ps(idx, ETALE_PH_SEED, st);
        etale_status s0 = seed_batch(idx, d, idx->x + (size_t)first * idx->mp, b, L, as<u64>(idx->seed),
                                     idx->insert_prec, st, idx->writer_sms, &rekey);
        if (s0 != ETALE_OK) return s0;
    }
    {
        PhaseScope ps(idx, ETALE_PH_SEARCH_INSERT, st);
        CK(launch_search(d, idx->x + (size_t)first * idx->mp, b, L, H, 1, 0, nullptr, nullptr,
                         as<u64>(idx->exp_keys), as<u32>(idx->exp_count), as<u64>(idx->seed), fit_tuning(idx, L, idx->tune),
                         idx->writer_sms, st, idx->insert_prec, 4, nullptr, idx->insert_prec == 0 && exact_rows(idx),
                         nullptr, nullptr, 0, rekey),
           "insert search");
    }
    g_kernel_launches += 1;
    // 2. forward edges, own slab, offers
    etale_status s = ensure_pool(idx, b, st);
    if (s != ETALE_OK) return s;
    {
        PhaseScope ps(idx, ETALE_PH_PRUNE, st);
        CK(launch_prune_insert(d, first, b, as<u64>(idx->exp_keys), as<u32>(idx->exp_count), H, idx->cfg.max_cand,
                               as<u32>(idx->F_id), as<float>(idx->F_rho), as<u32>(idx->F_n), of, idx->writer_sms, st,
                               idx->insert_prec != 0),
           "prune insert");
    }
    g_kernel_launches++;
    s = recycle(idx, st);
    if (s != ETALE_OK) return s;
    // 3. reverse offers (targets are nodes that existed before the sub-batch)
    s = run_offers(idx, slots, idx->live, st);
    if (s != ETALE_OK) return s;
    // 4. refine pass
    const u32 rmode = idx->cfg.refine == 1 ? 0 : idx->cfg.refine;
    if (rmode) {
        s = ensure_pool(idx, b, st);
        if (s != ETALE_OK) return s;
        {
            PhaseScope ps(idx, ETALE_PH_REFINE, st);
            const size_t sb = refine_spill_bytes(d, idx->cfg.max_cand, idx->writer_sms);
            if (!grow(idx->refine_spill, sb)) return idx->fail(ETALE_ENOMEM, "refine spill lists");
            CK(launch_refine(d, first, b, rmode, idx->cfg.max_cand, of, idx->writer_sms, st,
                             static_cast<char *>(idx->refine_spill.p), sb),
               "refine");
        }
        g_kernel_launches++;
        s = recycle(idx, st);
        if (s != ETALE_OK) return s;
        s = run_offers(idx, slots, idx->live + b, st);
        if (s != ETALE_OK) return s;
    }
    return ETALE_OK;
}

struct StreamCopy {
    // stage host inputs to device memory
    static etale_status in(etale_index *idx, DevBuf &buf, const void *src, size_t bytes, const void **dev,
                           cudaStream_t st) {
        if (is_device_ptr(src)) {
            *dev = src;
            return ETALE_OK;
        }
        if (!grow(buf, bytes)) return idx->fail(ETALE_ENOMEM, "staging allocation of %zu bytes", bytes);
        CK(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, st), "copy input");
        *dev = buf.p;
        return ETALE_OK;
    }
};

}  // namespace

struct etale_search_graph {
    etale_index *idx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float *qpad = nullptr;
    u64 *seed = nullptr;
    // tensor-core seeding: the graph's own query-side staging; the entry
    // copies are the index's, pinned while the graph lives
    bool tc = false;
    u32 S = 0;                            // |E| recorded
    void *tA = nullptr;
    float *tqstat = nullptr, *tkeys = nullptr;
    u32 *tfb = nullptr, *tctr = nullptr;
    u32 launches = 3;                     // kernels per replay
};

// ===========================================================================
extern "C" {

etale_status etale_config_default(etale_config *cfg) {
    if (!cfg) return ETALE_EINVAL;
    memset(cfg, 0, sizeof *cfg);
    cfg->build_beam = 64;
    cfg->alpha = 1.2f;
    cfg->refine = 2;
    cfg->n_entry = 1024;
    cfg->mode = ETALE_MODE_DETERMINISTIC;
    cfg->cas_budget = 16;
    cfg->rerank = 4;
    return ETALE_OK;
}

etale_status etale_create(uint32_t dim, etale_metric metric, uint32_t degree, uint64_t capacity,
                          const etale_config *cfg_in, etale_index **out) {
    if (!out) { t_last_error = "out is NULL"; return ETALE_EINVAL; }
    *out = nullptr;
    if (dim == 0 || degree == 0 || degree > (u32)MAX_R || capacity == 0 || capacity >= 0xFFFFFFFFull ||
        (metric != ETALE_L2 && metric != ETALE_IP)) {
        t_last_error = "invalid dim, metric, degree (1..64) or capacity";
        return ETALE_EINVAL;
    }
    etale_config cfg;
    etale_config_default(&cfg);
    if (cfg_in) {
        if (cfg_in->build_beam) cfg.build_beam = cfg_in->build_beam;
        if (cfg_in->alpha > 0.f) cfg.alpha = cfg_in->alpha;
        cfg.max_hops = cfg_in->max_hops;
        cfg.max_cand = cfg_in->max_cand;
        if (cfg_in->refine) cfg.refine = cfg_in->refine;
        cfg.max_batch = cfg_in->max_batch;
        cfg.pool_slabs = cfg_in->pool_slabs;
        if (cfg_in->n_entry) cfg.n_entry = cfg_in->n_entry;
        cfg.mode = cfg_in->mode;
        if (cfg_in->cas_budget) cfg.cas_budget = cfg_in->cas_budget;
        cfg.stage_kb = cfg_in->stage_kb;
        cfg.gram = cfg_in->gram;
        cfg.copies = cfg_in->copies;
        if (cfg_in->rerank) cfg.rerank = cfg_in->rerank;
        cfg.gt = cfg_in->gt;
        cfg.seed = cfg_in->seed;
        cfg.exact_rows = cfg_in->exact_rows;
    }
    if (cfg.gt > 1 || cfg.seed > 1 || cfg.exact_rows > 1) {
        t_last_error = "gt, seed and exact_rows must be 0 or 1";
        return ETALE_EINVAL;
    }
    if (cfg.copies > 3) {
        t_last_error = "copies is a bitmask of 1 (bf16) and 2 (fp8)";
        return ETALE_EINVAL;
    }
    if (cfg.gram > 2) {
        t_last_error = "gram must be 0..2";
        return ETALE_EINVAL;
    }
    if (cfg.gram == 0) cfg.gram = cfg.mode == ETALE_MODE_LOCKFREE ? 2 : 1;
    // the Gram tiles stage their rows from the bf16 copy
    if (cfg.gram == 2) cfg.copies |= 1u;
    if (cfg.stage_kb > 64) {
        t_last_error = "stage_kb must be <= 64";
        return ETALE_EINVAL;
    }
    if (cfg.refine > 2 || cfg.mode > 1 || cfg.build_beam > 256) {
        t_last_error = "refine must be 0..2, mode 0..1, build_beam <= 256";
        return ETALE_EINVAL;
    }
    if (cfg.max_cand == 0) cfg.max_cand = 2 * cfg.build_beam;
    if (cfg.max_batch == 0) cfg.max_batch = capacity / 100 ? capacity / 100 : 1;
    if (cfg.pool_slabs == 0) cfg.pool_slabs = 2 * capacity + 4ull * (degree + 1) * cfg.max_batch;
    if (cfg.pool_slabs >= 0xFFFFFFFFull) {
        t_last_error = "pool_slabs must be below 2^32 - 1";
        return ETALE_EINVAL;
    }
    etale_index *idx = new etale_index();
    idx->cfg = cfg;
    idx->seed_tc = cfg.seed == 0 && seed_tc_plan(dim, cfg.n_entry, 0).usable;
    idx->dim = dim;
    idx->mp = (dim + 3) / 4 * 4;
    idx->R = degree;
    idx->metric = (u32)metric;
    idx->capacity = capacity;
    idx->pool = cfg.pool_slabs;
    idx->alpha2 = cfg.alpha * cfg.alpha;
    cudaGetDevice(&idx->device);
    cudaDeviceGetAttribute(&idx->num_sms, cudaDevAttrMultiProcessorCount, idx->device);
    idx->writer_sms = idx->num_sms;
    cudaDeviceGetAttribute(&idx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, idx->device);
    const size_t xb = (size_t)capacity * idx->mp * 4, rb = (size_t)capacity * 8;
    const size_t sb = (size_t)idx->pool * degree * 8, pb = (size_t)idx->pool * 4;
    bool ok = cudaMalloc(&idx->x, xb) == cudaSuccess && cudaMalloc(&idx->ref, rb) == cudaSuccess &&
              cudaMalloc(&idx->slab, sb) == cudaSuccess && cudaMalloc(&idx->free_stack, pb) == cudaSuccess &&
              cudaMalloc(&idx->retired, pb) == cudaSuccess &&
              cudaMalloc(&idx->ctr, C_NCTR * sizeof(u64)) == cudaSuccess &&
              cudaMalloc(&idx->entries, (size_t)cfg.n_entry * 4) == cudaSuccess &&
              cudaMallocHost(&idx->host_ctr, C_NCTR * sizeof(u64)) == cudaSuccess &&
              cudaMallocHost(&idx->host_ctr_s, C_NCTR * sizeof(u64)) == cudaSuccess &&
              cudaMallocHost(&idx->host_ctr_st, C_NCTR * sizeof(u64)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&idx->stat_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&idx->search_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&idx->search_ev2, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&idx->nent_dev, 16) == cudaSuccess && cudaMemset(idx->nent_dev, 0, 16) == cudaSuccess &&
              cudaMalloc(&idx->rs, RS_N * sizeof(u64)) == cudaSuccess &&
              cudaMemset(idx->rs, 0, RS_N * sizeof(u64)) == cudaSuccess &&
              cudaEventCreateWithFlags(&idx->graph_ev, cudaEventDisableTiming) == cudaSuccess;
    idx->mb = (idx->mp + 7) / 8 * 8;
    idx->m8 = (idx->mp + 15) / 16 * 16;
    if (ok && (cfg.copies & 1))
        ok = cudaMalloc(&idx->xb, (size_t)capacity * idx->mb * 2) == cudaSuccess &&
             cudaMalloc(&idx->xbn, (size_t)capacity * 4) == cudaSuccess;
    if (ok && (cfg.copies & 2))
        ok = cudaMalloc(&idx->x8, (size_t)capacity * idx->m8) == cudaSuccess &&
             cudaMalloc(&idx->x8s, (size_t)capacity * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        t_last_error = "device allocation failed";
        etale_destroy(idx);
        return ETALE_ENOMEM;
    }
    idx->device_bytes = xb + rb + sb + 2 * pb + (idx->xb ? (size_t)capacity * (idx->mb * 2 + 4) : 0) +
                        (idx->x8 ? (size_t)capacity * (idx->m8 + 4) : 0);
    // refs <- <0, 0, NIL>; free stack <- all slabs; counters
    std::vector<u64> ctr(C_NCTR, 0);
    ctr[C_FREE] = idx->pool;
    bool ok2 = cudaMemset(idx->ref, 0, rb) == cudaSuccess;
    {
        // NIL slab field: low 32 bits all ones
        std::vector<u64> chunk(1 << 20, ref_pack(0, 0, NIL));
        for (size_t o = 0; o < capacity && ok2; o += chunk.size()) {
            size_t n = std::min(chunk.size(), (size_t)(capacity - o));
            ok2 = cudaMemcpy(idx->ref + o, chunk.data(), n * 8, cudaMemcpyHostToDevice) == cudaSuccess;
        }
        std::vector<u32> fs(1 << 20);
        for (size_t o = 0; o < idx->pool && ok2; o += fs.size()) {
            size_t n = std::min(fs.size(), (size_t)(idx->pool - o));
            for (size_t i = 0; i < n; i++) fs[i] = (u32)(idx->pool - 1 - (o + i));
            ok2 = cudaMemcpy(idx->free_stack + o, fs.data(), n * 4, cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    ok2 = ok2 && cudaMemcpy(idx->ctr, ctr.data(), C_NCTR * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
          cudaMemset(idx->x, 0, xb) == cudaSuccess;
    if (!ok2) {
        t_last_error = std::string("device initialisation failed: ") + cudaGetErrorString(cudaGetLastError());
        etale_destroy(idx);
        return ETALE_ECUDA;
    }
    idx->free_lb = idx->pool;
    *out = idx;
    return ETALE_OK;
}

etale_status etale_destroy(etale_index *idx) {
    if (!idx) return ETALE_OK;
    if (idx->round_graphs) {
        t_last_error = "destroy the index's round graphs and tensor-seeded query graphs first";
        return ETALE_EINVAL;
    }
    cudaFree(idx->x); cudaFree(idx->ref); cudaFree(idx->slab); cudaFree(idx->free_stack);
    cudaFree(idx->retired); cudaFree(idx->ctr); cudaFree(idx->entries);
    cudaFree(idx->xb); cudaFree(idx->xbn); cudaFree(idx->x8); cudaFree(idx->x8s); cudaFree(idx->nent_dev); cudaFree(idx->rs);
    if (idx->graph_ev) cudaEventDestroy(idx->graph_ev);
    if (idx->host_ctr) cudaFreeHost(idx->host_ctr);
    if (idx->host_ctr_s) cudaFreeHost(idx->host_ctr_s);
    if (idx->host_ctr_st) cudaFreeHost(idx->host_ctr_st);
    if (idx->stat_stream) cudaStreamDestroy(idx->stat_stream);
    if (idx->search_ev) cudaEventDestroy(idx->search_ev);
    if (idx->search_ev2) cudaEventDestroy(idx->search_ev2);
    for (cudaEvent_t e : idx->pev) cudaEventDestroy(e);
    DevBuf *bufs[] = {&idx->stage, &idx->qpad, &idx->out_ids, &idx->out_dist, &idx->exp_keys, &idx->exp_count,
                      &idx->F_id, &idx->F_rho, &idx->F_n, &idx->of_key, &idx->of_val, &idx->of_key2,
                      &idx->of_val2, &idx->of_src, &idx->of_rho, &idx->seg_flags, &idx->seg_scan, &idx->seg_start,
                      &idx->sort_scr, &idx->scan_scr, &idx->live_flags, &idx->live_rank, &idx->live_scan_scr,
                      &idx->tomb_bits, &idx->del_ids, &idx->del_vals, &idx->del_ids2, &idx->del_vals2,
                      &idx->del_ok, &idx->del_scan, &idx->dt, &idx->pair_key, &idx->pair_val, &idx->pair_key2,
                      &idx->pair_val2, &idx->pair_K, &idx->pair_Kn, &idx->pair_flags, &idx->pair_scan,
                      &idx->pair_seg, &idx->counts, &idx->ex_del, &idx->ex_hs, &idx->ex_deg, &idx->ex_ids,
                      &idx->ex_rho, &idx->seed, &idx->s_stage, &idx->s_qpad, &idx->s_out_ids, &idx->s_out_dist,
                      &idx->s_seed};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete idx;
    return ETALE_OK;
}

etale_status etale_insert(etale_index *idx, const float *vecs, uint64_t n, uint32_t *out_ids, void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (n == 0) return ETALE_OK;
    if (!vecs) return idx->fail(ETALE_EINVAL, "vecs is NULL");
    if (idx->next_id + n > idx->capacity)
        return idx->fail(ETALE_ECAPACITY, "insert of %llu would exceed capacity %llu (next id %llu)",
                         (unsigned long long)n, (unsigned long long)idx->capacity, (unsigned long long)idx->next_id);
    cudaStream_t st = (cudaStream_t)stream;
    etale_status s = writer_begin(idx, st);
    if (s != ETALE_OK) return s;
    {
        // before any change: the largest phase of the largest sub-batch must
        // fit the pool (each insert publishes at most 1 + R times per phase)
        const u64 b = std::min<u64>(n, idx->cfg.max_batch);
        s = ensure_pool(idx, b * (idx->R + 1), st);
        if (s != ETALE_OK) return s;
        idx->free_lb += b * (idx->R + 1);
    }
    const void *src = nullptr;
    s = StreamCopy::in(idx, idx->stage, vecs, (size_t)n * idx->dim * 4, &src, st);
    if (s != ETALE_OK) return s;
    const u64 first_all = idx->next_id;
    CK(launch_ingest(idx->x + first_all * idx->mp, idx->mp, (const float *)src, idx->dim, n, st), "ingest");
    CK(launch_ingest_copies(idx->dev(), first_all, n, st), "ingest copies");
    g_kernel_launches += 2;
    if (idx->rows_exact && idx->xb && idx->cfg.exact_rows == 1) {
        // the batch's searches below gather the bf16 copy only if it is still exact
        s = read_ctr(idx, st);
        if (s != ETALE_OK) return s;
        idx->rows_exact = idx->host_ctr[C_INEXACT] == 0;
    }
    u64 done = 0;
    const u64 maxb = idx->cfg.max_batch;
    s = size_batch_scratch(idx, std::min<u64>(n, maxb));
    if (s != ETALE_OK) return s;
    while (done < n) {
        u64 b = n - done;
        const u64 cap = idx->live ? idx->live : 1;
        if (b > cap) b = cap;
        if (b > maxb) b = maxb;
        const u32 first = (u32)idx->next_id;
        idx->next_id += b;
        s = insert_subbatch(idx, first, (u32)b, st);
        if (s != ETALE_OK) return s;
        idx->live += b;
        s = recompute_entries(idx, st);
        if (s != ETALE_OK) return s;
        done += b;
    }
    std::vector<u32> ids;
    if (out_ids) {
        ids.resize(n);
        for (u64 i = 0; i < n; i++) ids[i] = (u32)(first_all + i);
        CK(cudaMemcpyAsync(out_ids, ids.data(), n * 4, cudaMemcpyDefault, st), "write ids");
    }
    return check_device_errors(idx, st);   // synchronises before `ids` goes away
}

etale_status etale_delete(etale_index *idx, const uint32_t *ids, uint64_t n, uint64_t *n_deleted, void *stream) {
    if (!idx) return ETALE_EINVAL;
    if (n_deleted) *n_deleted = 0;
    if (n == 0) return ETALE_OK;
    if (!ids) return idx->fail(ETALE_EINVAL, "ids is NULL");
    if (n > 0x7FFFFFFFull / MAX_R) return idx->fail(ETALE_EINVAL, "delete batch too large");
    cudaStream_t st = (cudaStream_t)stream;
    {
        etale_status s0 = settle(idx);
        if (s0 != ETALE_OK) return s0;
    }
    const u32 R = idx->R;
    const u64 slots = n * R;
    if (!size_delete_scratch(idx, n))
        return idx->fail(ETALE_ENOMEM, "scratch allocation (delete batch of %llu)", (unsigned long long)n);
    {
        etale_status sb = writer_begin(idx, st);
        if (sb != ETALE_OK) return sb;
    }
    if (is_device_ptr(ids)) {
        CK(cudaMemcpyAsync(idx->del_ids.p, ids, n * 4, cudaMemcpyDeviceToDevice, st), "copy ids");
    } else {
        CK(cudaMemcpyAsync(idx->del_ids.p, ids, n * 4, cudaMemcpyHostToDevice, st), "copy ids");
    }
    Dev d = idx->dev();
    SortScratch ss;
    sort_scratch_carve(ss, as<u32>(idx->sort_scr), (u32)std::max<u64>(slots, n));
    ScanScratch sc;
    scan_scratch_carve(sc, as<u32>(idx->scan_scr), (u32)std::max<u64>(slots, n));
    // sorted ids (payload unused)
    prof_begin(idx, ETALE_PH_DELETE_PREP, st);
    CK(launch_fill_offer_keys(as<u32>(idx->del_vals2), as<u32>(idx->del_vals), (u32)n, 0, st), "iota");
    CK(radix_sort_pairs(as<u32>(idx->del_ids), as<u32>(idx->del_vals), as<u32>(idx->del_ids2),
                        as<u32>(idx->del_vals2), (u32)n, 32, ss, st),
       "sort ids");
    u64 *n_dt = as<u64>(idx->counts) + 1;
    u64 *seg_count = as<u64>(idx->counts) + 2;
    CK(launch_tombstone(d, as<u32>(idx->del_ids), (u32)n, idx->next_id, as<u32>(idx->del_ok), st), "tombstone");
    CK(exclusive_scan(as<u32>(idx->del_ok), as<u32>(idx->del_scan), (u32)n, sc, st), "tombstone scan");
    CK(launch_compact_ok(as<u32>(idx->del_ids), as<u32>(idx->del_ok), as<u32>(idx->del_scan), (u32)n,
                         as<u32>(idx->dt), n_dt, st),
       "tombstone compaction");
    g_kernel_launches += 4 * 3 + 6;
    prof_end(idx, st);
    // repair: K(u, a) per pair, then one fold per a
    const u32 invalid = (u32)idx->capacity;
    prof_begin(idx, ETALE_PH_REPAIR_K, st);
    CK(launch_fill_offer_keys(as<u32>(idx->pair_key), as<u32>(idx->pair_val), (u32)slots, invalid, st), "fill pairs");
    CK(launch_repair_k(d, as<u32>(idx->dt), n_dt, (u32)n, as<u32>(idx->pair_key), as<u32>(idx->pair_val),
                       as<uint2>(idx->pair_K), as<u32>(idx->pair_Kn), idx->writer_sms, st),
       "repair K");
    g_kernel_launches += 2;
    prof_end(idx, st);
    const bool lockfree = idx->cfg.mode == ETALE_MODE_LOCKFREE;
    etale_status s = ETALE_OK;
    if (lockfree) {
        // one publication per (deleted, neighbour) pair: chunk as for offers
        for (u64 lo = 0; lo < slots;) {
            u64 chunk;
            s = lockfree_chunk(idx, slots - lo, &chunk, st);
            if (s != ETALE_OK) return s;
            prof_begin(idx, ETALE_PH_REPAIR_FOLD, st);
            CK(launch_repair_fold(d, as<u32>(idx->dt), as<u32>(idx->pair_key), as<u32>(idx->pair_val),
                                  as<uint2>(idx->pair_K), as<u32>(idx->pair_Kn), nullptr, seg_count, chunk,
                                  idx->cfg.cas_budget, idx->writer_sms, st, lo),
               "repair fold");
            g_kernel_launches++;
            prof_end(idx, st);
            s = recycle(idx, st);
            if (s != ETALE_OK) return s;
            lo += chunk;
        }
    }
    if (!lockfree) s = ensure_pool(idx, std::min<u64>(slots, idx->live), st);
    if (s != ETALE_OK) return s;
    if (!lockfree) prof_begin(idx, ETALE_PH_REPAIR_FOLD, st);
    if (!lockfree) {
        CK(radix_sort_pairs(as<u32>(idx->pair_key), as<u32>(idx->pair_val), as<u32>(idx->pair_key2),
                            as<u32>(idx->pair_val2), (u32)slots, bits_for(idx->capacity), ss, st),
           "pair sort");
        CK(make_segments(as<u32>(idx->pair_key), (u32)slots, invalid, as<u32>(idx->pair_flags),
                         as<u32>(idx->pair_scan), as<u32>(idx->pair_seg), seg_count, sc, st),
           "pair segments");
        g_kernel_launches += 3 * ((bits_for(idx->capacity) + 7) / 8) * 2 + 4;
    }
    if (!lockfree) {
        CK(launch_repair_fold(d, as<u32>(idx->dt), as<u32>(idx->pair_key), as<u32>(idx->pair_val),
                              as<uint2>(idx->pair_K), as<u32>(idx->pair_Kn), as<u32>(idx->pair_seg), seg_count, slots,
                              0, idx->writer_sms, st),
           "repair fold");
        g_kernel_launches++;
        prof_end(idx, st);
        s = recycle(idx, st);
        if (s != ETALE_OK) return s;
    }
    u64 k = 0;
    CK(cudaMemcpyAsync(&k, n_dt, sizeof k, cudaMemcpyDeviceToHost, st), "read count");
    s = check_device_errors(idx, st);   // synchronises
    idx->live -= k;
    idx->tombs += k;
    if (n_deleted) *n_deleted = k;
    return s;
}

etale_status etale_reclaim(etale_index *idx, void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    cudaStream_t st = (cudaStream_t)stream;
    etale_status s = writer_begin(idx, st);
    if (s != ETALE_OK) return s;
    s = recompute_entries(idx, st);
    if (s != ETALE_OK) return s;
    const u64 n = idx->next_id;
    if (n == 0) return check_device_errors(idx, st);
    if (!grow(idx->tomb_bits, ((n + 31) / 32) * 4)) return idx->fail(ETALE_ENOMEM, "scratch allocation (reclaim)");
    Dev d = idx->dev();
    s = ensure_pool(idx, idx->live, st);
    if (s != ETALE_OK) return s;
    {
        PhaseScope ps(idx, ETALE_PH_COMPACT, st);
        CK(launch_tomb_bits(d, n, as<u32>(idx->tomb_bits), st), "tombstone bitmap");
        CK(launch_compact(d, n, as<u32>(idx->tomb_bits), st), "compaction");
    }
    g_kernel_launches += 2;
    s = recycle(idx, st);
    if (s != ETALE_OK) return s;
    {
        PhaseScope ps(idx, ETALE_PH_RECLAIM, st);
        CK(launch_reclaim_tombstones(d, n, st), "reclaim");
    }
    g_kernel_launches++;
    s = recycle(idx, st);
    if (s != ETALE_OK) return s;
    s = check_device_errors(idx, st);
    idx->reclaimed += idx->tombs;
    idx->tombs = 0;
    return s;
}

// Tensor-core candidate pass + certified exact rerank; queries it cannot
// certify, and shapes it does not cover, run on the CUDA-core exact kernel.
static etale_status ground_truth_run(etale_index *idx, const Dev &d, const float *qpad, u32 nq, u32 k, u32 *oid,
                                     float *od, cudaStream_t st) {
    idx->gt_path = 0;
    idx->gt_fallbacks = 0;
    GtTcPlan p = gt_tc_plan(idx->dim, idx->next_id, nq);
    if (idx->cfg.gt == 1 || p.n_pad == 0) {
        PhaseScope ps(idx, ETALE_PH_GT_EXACT, st);
        CK(launch_ground_truth(d, idx->next_id, qpad, nq, k, oid, od, idx->num_sms, st), "ground truth");
        g_kernel_launches++;
        return ETALE_OK;
    }
    if (!grow(idx->gt_A, p.bytes_A) || !grow(idx->gt_B, p.bytes_B) || !grow(idx->gt_xn, p.n_pad * 4) ||
        !grow(idx->gt_qstat, (size_t)nq * 16) || !grow(idx->gt_gstat, 64) || !grow(idx->gt_fb, (size_t)nq * 4))
        return idx->fail(ETALE_ENOMEM, "ground-truth staging");
    GtTcBufs b{};
    b.A = idx->gt_A.p;
    b.B = idx->gt_B.p;
    b.xn = as<float>(idx->gt_xn);
    b.qstat = as<float>(idx->gt_qstat);
    b.gstat = as<u32>(idx->gt_gstat);
    b.fb = as<u32>(idx->gt_fb);
    b.err = b.gstat + 5;
    {
        PhaseScope ps(idx, ETALE_PH_GT_PREP, st);
        CK(launch_gt_tc_prep(d, idx->next_id, qpad, nq, p, b, st), "ground-truth copies");
    }
    g_kernel_launches += 2;
    u32 h[8];
    CK(cudaMemcpyAsync(h, b.gstat, sizeof h, cudaMemcpyDeviceToHost, st), "read split flag");
    CK(cudaStreamSynchronize(st), "synchronize");
    gt_tc_configure(p, nq, h[3] != 0);
    if (!p.usable) {
        PhaseScope ps(idx, ETALE_PH_GT_EXACT, st);
        CK(launch_ground_truth(d, idx->next_id, qpad, nq, k, oid, od, idx->num_sms, st), "ground truth");
        g_kernel_launches++;
        return ETALE_OK;
    }
    if (!grow(idx->gt_bmin, p.bytes_bmin)) return idx->fail(ETALE_ENOMEM, "ground-truth block minima");
    b.bmin = as<float>(idx->gt_bmin);
    for (u32 q0 = 0; q0 < nq; q0 += p.qgroup) {
        const u32 g = std::min<u32>(p.qgroup, nq - q0);
        {
            PhaseScope ps(idx, ETALE_PH_GT_TENSOR, st);
            CK(launch_gt_tc(d, q0, g, p, b, idx->next_id, idx->num_sms, st), "ground truth (tensor)");
        }
        {
            PhaseScope ps(idx, ETALE_PH_GT_MERGE, st);
            CK(launch_gt_rerank(d, qpad, q0, g, k, p, b, idx->next_id, oid, od, st), "ground truth (rerank)");
        }
        g_kernel_launches += 2;
    }
    CK(cudaMemcpyAsync(h, b.gstat, sizeof h, cudaMemcpyDeviceToHost, st), "read fallback count");
    CK(cudaStreamSynchronize(st), "synchronize");
    if (h[5] & ERR_TIMEOUT) return idx->fail(ETALE_ETIMEOUT, "ground truth: a bounded device wait gave up");
    idx->gt_path = p.split ? 2 : 1;
    idx->gt_fallbacks = h[4];
    if (h[4]) {
        PhaseScope ps(idx, ETALE_PH_GT_EXACT, st);
        CK(launch_ground_truth(d, idx->next_id, qpad, h[4], k, oid, od, idx->num_sms, st, b.fb),
           "ground truth (fallback)");
        g_kernel_launches++;
    }
    return ETALE_OK;
}

static etale_status search_common(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, uint32_t beam,
                                  uint32_t *out_ids, float *out_dists, void *stream, bool exact) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (nq == 0) return ETALE_OK;
    if (!queries || !out_ids || !out_dists || k == 0) return idx->fail(ETALE_EINVAL, "null buffer or k == 0");
    if (exact && k > 32) return idx->fail(ETALE_EINVAL, "ground truth supports k <= 32");
    const u32 L = beam > k ? beam : k;
    if (!exact && L > 256) return idx->fail(ETALE_EINVAL, "beam must be <= 256");
    if (!exact && idx->search_prec && k > 64) return idx->fail(ETALE_EINVAL, "reduced-precision search needs k <= 64");
    if (nq > 0xFFFFFFFFull) return idx->fail(ETALE_EINVAL, "too many queries");
    cudaStream_t st = (cudaStream_t)stream;
    const void *src = nullptr;
    etale_status s = StreamCopy::in(idx, idx->s_stage, queries, (size_t)nq * idx->dim * 4, &src, st);
    if (s != ETALE_OK) return s;
    if (!grow(idx->s_qpad, (size_t)nq * idx->mp * 4)) return idx->fail(ETALE_ENOMEM, "query staging");
    float *qpad = as<float>(idx->s_qpad);
    CK(launch_ingest(qpad, idx->mp, (const float *)src, idx->dim, nq, st), "query ingest");
    const bool dev_out = is_device_ptr(out_ids) && is_device_ptr(out_dists);
    u32 *oid = out_ids;
    float *od = out_dists;
    if (!dev_out) {
        if (!grow(idx->s_out_ids, nq * k * 4) || !grow(idx->s_out_dist, nq * k * 4))
            return idx->fail(ETALE_ENOMEM, "output staging");
        oid = as<u32>(idx->s_out_ids);
        od = as<float>(idx->s_out_dist);
    }
    Dev d = idx->dev();
    const bool prof = idx->prof && !idx->concurrent;
    if (exact) {
        s = ground_truth_run(idx, d, qpad, (u32)nq, k, oid, od, st);
        if (s != ETALE_OK) return s;
    } else {
        const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * L;
        if (!grow(idx->s_seed, (size_t)nq * L * 8)) return idx->fail(ETALE_ENOMEM, "seed buffer");
        if (prof) prof_begin(idx, ETALE_PH_SEED, st);
        bool rekey = false;
        s = seed_batch(idx, d, qpad, (u32)nq, L, as<u64>(idx->s_seed), idx->search_prec, st, 0, &rekey);
        if (prof) prof_end(idx, st);
        if (s != ETALE_OK) return s;
        if (prof) prof_begin(idx, ETALE_PH_SEARCH_QUERY, st);
        CK(launch_search(d, qpad, (u32)nq, L, H, 0, k, oid, od, nullptr, nullptr, as<u64>(idx->s_seed), fit_tuning(idx, L, idx->tune),
                         idx->num_sms, st, idx->search_prec, idx->cfg.rerank, nullptr,
                         idx->search_prec == 0 && exact_rows(idx), nullptr, nullptr, 0, rekey),
           "search");
        if (prof) prof_end(idx, st);
        g_kernel_launches++;
        if (idx->concurrent) {
            std::lock_guard<std::mutex> lk(idx->mu);
            CK(cudaEventRecord(idx->search_ev, st), "record search event");
            idx->search_ev_valid = true;
        }
    }
    g_kernel_launches++;       // query ingest
    if (!dev_out) {
        CK(cudaMemcpyAsync(out_ids, oid, nq * k * 4, cudaMemcpyDeviceToHost, st), "copy ids out");
        CK(cudaMemcpyAsync(out_dists, od, nq * k * 4, cudaMemcpyDeviceToHost, st), "copy dists out");
    }
    return check_search_errors(idx, st);
}

etale_status etale_search(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, uint32_t beam,
                          uint32_t *out_ids, float *out_dists, void *stream) {
    return search_common(idx, queries, nq, k, beam, out_ids, out_dists, stream, false);
}

etale_status etale_search_eval_count(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, uint32_t beam,
                                     uint64_t *n_eval, uint64_t *n_unique, uint64_t *n_expand, void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (!queries || !n_eval || !n_unique || !n_expand || k == 0 || nq == 0)
        return idx->fail(ETALE_EINVAL, "null argument, k == 0 or nq == 0");
    const u32 L = beam > k ? beam : k;
    if (L > 256 || nq > 0xFFFFFFFFull) return idx->fail(ETALE_EINVAL, "beam must be <= 256");
    if (idx->search_prec && k > 64) return idx->fail(ETALE_EINVAL, "reduced-precision search needs k <= 64");
    const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * L;
    const u64 cap = (u64)H * idx->R;   // no search evaluates more (one slab per expansion)
    if (cap > (1u << 15) || eval_unique_smem((u32)cap, L) > (size_t)idx->smem_optin)
        return idx->fail(ETALE_EINVAL, "evaluation log of %llu ids per query is above 32768",
                         (unsigned long long)cap);
    cudaStream_t st = (cudaStream_t)stream;
    const void *src = nullptr;
    etale_status s = StreamCopy::in(idx, idx->s_stage, queries, (size_t)nq * idx->dim * 4, &src, st);
    if (s != ETALE_OK) return s;
    float *qpad = nullptr;
    u64 *seed = nullptr, *cnt = nullptr;
    u32 *elog = nullptr, *elog_n = nullptr, *oid = nullptr;
    float *od = nullptr;
    cudaError_t e = cudaMalloc(&qpad, (size_t)nq * idx->mp * 4);
    if (e == cudaSuccess) e = cudaMalloc(&seed, (size_t)nq * L * 8);
    if (e == cudaSuccess) e = cudaMalloc(&elog, (size_t)nq * cap * 4);
    if (e == cudaSuccess) e = cudaMalloc(&elog_n, (size_t)nq * 4);
    if (e == cudaSuccess) e = cudaMalloc(&oid, (size_t)nq * k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&od, (size_t)nq * k * 4);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, 4 * 8);
    u64 h[4] = {0, 0, 0, 0}, e0 = 0, e1 = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4 * 8, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&e0, idx->ctr + C_EXPAND, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = launch_ingest(qpad, idx->mp, (const float *)src, idx->dim, nq, st);
    Dev d = idx->dev();
    if (e == cudaSuccess) e = launch_seed(d, qpad, (u32)nq, L, seed, st, idx->search_prec);
    if (e == cudaSuccess)
        e = launch_search(d, qpad, (u32)nq, L, H, 0, k, oid, od, nullptr, nullptr, seed, fit_tuning(idx, L, idx->tune),
                          idx->num_sms, st, idx->search_prec, idx->cfg.rerank, nullptr,
                          idx->search_prec == 0 && exact_rows(idx), elog, elog_n, (u32)cap);
    const u32 n0 = std::min<u32>(L, idx->n_entries);
    if (e == cudaSuccess) e = launch_eval_unique(elog, elog_n, (u32)cap, seed, L, n0, (u32)nq, cnt, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, cnt, 4 * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&e1, idx->ctr + C_EXPAND, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    g_kernel_launches += 4;
    cudaFree(qpad); cudaFree(seed); cudaFree(elog); cudaFree(elog_n); cudaFree(oid); cudaFree(od); cudaFree(cnt);
    if (e != cudaSuccess) return idx->cuda_fail(e, "evaluation count");
    if (h[2]) return idx->fail(ETALE_EINTERNAL, "evaluation log overflowed");
    *n_eval = h[0];
    *n_unique = h[1];
    *n_expand = e1 - e0;
    return check_search_errors(idx, st);
}

etale_status etale_ground_truth(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, uint32_t *out_ids,
                                float *out_dists, void *stream) {
    return search_common(idx, queries, nq, k, 0, out_ids, out_dists, stream, true);
}

etale_status etale_export_graph(etale_index *idx, uint64_t n, uint8_t *deleted, uint8_t *has_slab, uint8_t *degree,
                                uint32_t *nbr_ids, float *nbr_rho, void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (n > idx->next_id) return idx->fail(ETALE_EINVAL, "n exceeds next_id");
    if (n == 0) return ETALE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const u64 R = idx->R;
    if (!grow(idx->ex_del, n) || !grow(idx->ex_hs, n) || !grow(idx->ex_deg, n) || !grow(idx->ex_ids, n * R * 4) ||
        !grow(idx->ex_rho, n * R * 4))
        return idx->fail(ETALE_ENOMEM, "export staging");
    CK(launch_export(idx->dev(), n, as<unsigned char>(idx->ex_del), as<unsigned char>(idx->ex_hs),
                     as<unsigned char>(idx->ex_deg), as<u32>(idx->ex_ids), as<float>(idx->ex_rho), st),
       "export");
    g_kernel_launches++;
    CK(cudaMemcpyAsync(deleted, idx->ex_del.p, n, cudaMemcpyDefault, st), "export copy");
    CK(cudaMemcpyAsync(has_slab, idx->ex_hs.p, n, cudaMemcpyDefault, st), "export copy");
    CK(cudaMemcpyAsync(degree, idx->ex_deg.p, n, cudaMemcpyDefault, st), "export copy");
    CK(cudaMemcpyAsync(nbr_ids, idx->ex_ids.p, n * R * 4, cudaMemcpyDefault, st), "export copy");
    CK(cudaMemcpyAsync(nbr_rho, idx->ex_rho.p, n * R * 4, cudaMemcpyDefault, st), "export copy");
    CK(cudaStreamSynchronize(st), "synchronize");
    return ETALE_OK;
}

etale_status etale_get_entries(etale_index *idx, uint32_t *out, uint32_t *n) {
    if (!idx || !out || !n) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    *n = idx->n_entries;
    if (idx->n_entries == 0) return ETALE_OK;
    cudaError_t e = cudaMemcpy(out, idx->entries, (size_t)idx->n_entries * 4, cudaMemcpyDefault);
    return e == cudaSuccess ? ETALE_OK : idx->cuda_fail(e, "copy entries");
}

etale_status etale_stats(etale_index *idx, etale_stats_t *o) {
    if (!idx || !o) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    // a private non-blocking stream: reading the counters never waits for,
    // or orders against, the caller's streams
    cudaError_t e = cudaMemcpyAsync(idx->host_ctr_st, idx->ctr, C_NCTR * sizeof(u64), cudaMemcpyDeviceToHost,
                                    idx->stat_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(idx->stat_stream);
    if (e != cudaSuccess) return idx->cuda_fail(e, "read counters");
    memset(o, 0, sizeof *o);
    const u64 *c = idx->host_ctr_st;
    o->live = idx->live;
    o->tombstones = idx->tombs;
    o->reclaimed = idx->reclaimed;
    o->next_id = idx->next_id;
    o->capacity = idx->capacity;
    o->pool_slabs = idx->pool;
    o->free_slabs = c[C_FREE] - std::min(c[C_POP], c[C_FREE]);
    o->retired_slabs = c[C_RET];
    o->used_slabs = idx->pool - o->free_slabs - o->retired_slabs;
    o->n_entries = idx->n_entries;
    o->degree = idx->R;
    o->n_publish = c[C_PUBLISH];
    o->n_cas_retry = c[C_CAS_RETRY];
    o->n_dropped = c[C_DROPPED];
    o->n_expand = c[C_EXPAND];
    o->n_dist = c[C_DIST];
    o->device_bytes = idx->device_bytes;
    o->exact_rows = exact_rows(idx) ? 1 : 0;
    o->dim = idx->dim;
    o->metric = idx->metric;
    return ETALE_OK;
}

etale_status etale_get_config(const etale_index *idx, etale_config *out) {
    if (!idx || !out) return ETALE_EINVAL;
    *out = idx->cfg;
    return ETALE_OK;
}

const char *etale_last_error(const etale_index *) { return t_last_error.c_str(); }

etale_status etale_set_exact_rows(etale_index *idx, int on) {
    if (!idx) return ETALE_EINVAL;
    if (on && idx->rows_exact && idx->xb) {
        // rows ingested while the gathers were off were counted on the device
        u64 inexact = 0;
        CK(cudaMemcpy(&inexact, idx->ctr + C_INEXACT, sizeof inexact, cudaMemcpyDeviceToHost), "read counter");
        idx->rows_exact = inexact == 0;
    }
    idx->cfg.exact_rows = on ? 1u : 0u;
    return ETALE_OK;
}

etale_status etale_set_search_tuning(etale_index *idx, uint32_t stage_rows, uint32_t seen_bits,
                                     uint32_t warps_per_block) {
    if (!idx) return ETALE_EINVAL;
    if (stage_rows < 1 || stage_rows > 32 || seen_bits < 6 || seen_bits > 14)
        return idx->fail(ETALE_EINVAL, "stage_rows must be 1..32 and seen_bits 6..14");
    if (warps_per_block && warps_per_block != 2 && warps_per_block != 4 && warps_per_block != 8)
        return idx->fail(ETALE_EINVAL, "warps_per_block must be 2, 4 or 8 (0 keeps it)");
    idx->tune.stage_rows = stage_rows;
    idx->tune.seen_bits = seen_bits;
    if (warps_per_block) idx->tune.warps_per_block = warps_per_block;
    return ETALE_OK;
}

etale_status etale_set_search_keys(etale_index *idx, int tensor) {
    if (!idx) return ETALE_EINVAL;
    if (tensor != 0 && tensor != 1) return idx->fail(ETALE_EINVAL, "tensor must be 0 or 1");
    idx->tune.keys_tc = (u32)tensor;
    return ETALE_OK;
}

etale_status etale_autotune_search(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, uint32_t beam,
                                   etale_tuning *out, uint32_t n_out, uint32_t *n_tried, void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (n_tried) *n_tried = 0;
    if (!queries || nq == 0 || k == 0 || !is_device_ptr(queries))
        return idx->fail(ETALE_EINVAL, "autotune needs a non-empty DEVICE query batch");
    const u32 L = beam > k ? beam : k;
    if (L > 256 || nq > 0xFFFFFFFFull) return idx->fail(ETALE_EINVAL, "beam must be <= 256");
    cudaStream_t st = (cudaStream_t)stream;
    if (!grow(idx->s_qpad, (size_t)nq * idx->mp * 4) || !grow(idx->s_seed, (size_t)nq * L * 8) ||
        !grow(idx->s_out_ids, nq * k * 4) || !grow(idx->s_out_dist, nq * k * 4))
        return idx->fail(ETALE_ENOMEM, "autotune scratch");
    float *qpad = as<float>(idx->s_qpad);
    CK(launch_ingest(qpad, idx->mp, queries, idx->dim, nq, st), "query ingest");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const SearchTuning saved = idx->tune;
    const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * L;
    float best = 1e30f;
    SearchTuning best_t = saved;
    u32 tried = 0;
    const u32 rows[4] = {2, 4, 8, 16}, bits[4] = {7, 8, 9, 10}, wpbs[3] = {2, 4, 8};
    // BF16 searches also try both key paths (tensor cores, CUDA cores)
    const u32 n_keys = idx->search_prec == 1 ? 2u : 1u;
    for (u32 kp = 0; kp < n_keys; kp++)
    for (u32 c = 0; c < 3; c++)
    for (u32 a = 0; a < 4; a++)
        for (u32 b = 0; b < 4; b++) {
            SearchTuning t;
            t.stage_rows = rows[a];
            t.seen_bits = bits[b];
            t.warps_per_block = wpbs[c];
            t.keys_tc = kp == 0 ? 1u : 0u;
            if (fit_tuning(idx, L, t).stage_rows != t.stage_rows) continue;   // does not fit: not a shape
            float ms_best = 1e30f;
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; rep++) {   // first run warms up
                Dev d = idx->dev();
                cudaEventRecord(e0, st);
                ok = launch_seed(d, qpad, (u32)nq, L, as<u64>(idx->s_seed), st, idx->search_prec) == cudaSuccess &&
                     launch_search(d, qpad, (u32)nq, L, H, 0, k, as<u32>(idx->s_out_ids), as<float>(idx->s_out_dist),
                                   nullptr, nullptr, as<u64>(idx->s_seed), t, idx->num_sms, st, idx->search_prec,
                                   idx->cfg.rerank, nullptr, idx->search_prec == 0 && exact_rows(idx)) == cudaSuccess;
                cudaEventRecord(e1, st);
                if (cudaStreamSynchronize(st) != cudaSuccess) ok = false;
                float ms = 0.f;
                if (ok && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms_best = std::min(ms_best, ms);
            }
            cudaGetLastError();   // a shape that does not fit is skipped
            if (!ok) continue;
            if (out && tried < n_out)
                out[tried] = etale_tuning{t.stage_rows, t.seen_bits, ms_best, t.warps_per_block, t.keys_tc};
            tried++;
            if (ms_best < best) { best = ms_best; best_t = t; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_kernel_launches += 1 + 2 * 3 * tried;
    idx->tune = tried ? best_t : saved;
    if (n_tried) *n_tried = tried;
    return check_search_errors(idx, st);
}

etale_status etale_autotune_beam(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, float target,
                                 const uint32_t *beams, uint32_t n_beams, float *recalls, uint32_t *chosen,
                                 void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (!queries || !is_device_ptr(queries) || nq == 0 || nq > 0xFFFFFFFFull || k == 0 || k > 32 || !beams ||
        n_beams == 0 || !chosen)
        return idx->fail(ETALE_EINVAL, "autotune_beam needs a DEVICE query batch, k in 1..32 and beams");
    for (u32 i = 0; i < n_beams; i++)
        if (beams[i] > 256 || (i && beams[i] <= beams[i - 1]))
            return idx->fail(ETALE_EINVAL, "beams must ascend and stay <= 256");
    const size_t nk = (size_t)nq * k;
    u32 *gid = nullptr, *sid = nullptr;
    float *gd = nullptr, *sd = nullptr;
    if (cudaMalloc(&gid, nk * 4) != cudaSuccess || cudaMalloc(&sid, nk * 4) != cudaSuccess ||
        cudaMalloc(&gd, nk * 4) != cudaSuccess || cudaMalloc(&sd, nk * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(gid); cudaFree(sid); cudaFree(gd); cudaFree(sd);
        return idx->fail(ETALE_ENOMEM, "autotune_beam buffers");
    }
    std::vector<u32> gh(nk), sh(nk);
    etale_status s = search_common(idx, queries, nq, k, 0, gid, gd, stream, true);   // exact top-k
    if (s == ETALE_OK && cudaMemcpy(gh.data(), gid, nk * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        s = idx->fail(ETALE_ECUDA, "autotune_beam copy");
    for (u32 i = 0; i < n_beams; i++) recalls ? (void)(recalls[i] = -1.0f) : (void)0;
    u32 pick = beams[n_beams - 1];
    for (u32 i = 0; i < n_beams && s == ETALE_OK; i++) {
        s = search_common(idx, queries, nq, k, beams[i], sid, sd, stream, false);
        if (s != ETALE_OK) break;
        if (cudaMemcpy(sh.data(), sid, nk * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            s = idx->fail(ETALE_ECUDA, "autotune_beam copy");
            break;
        }
        u64 hit = 0;
        for (u64 q = 0; q < nq; q++) {
            const u32 *a = sh.data() + q * k, *b = gh.data() + q * k;
            for (u32 x = 0; x < k; x++) {
                if (a[x] == NIL) continue;
                for (u32 y = 0; y < k; y++)
                    if (a[x] == b[y]) { hit++; break; }
            }
        }
        const float rec = (float)((double)hit / (double)nk);
        if (recalls) recalls[i] = rec;
        if (rec >= target) {
            pick = beams[i];
            break;
        }
    }
    cudaFree(gid); cudaFree(sid); cudaFree(gd); cudaFree(sd);
    if (s != ETALE_OK) return s;
    *chosen = pick;
    return etale_autotune_search(idx, queries, nq, k, pick, nullptr, 0, nullptr, stream);
}

etale_status etale_search_graph_create(etale_index *idx, uint32_t nq_max, uint32_t k, uint32_t beam,
                                       const float *queries, uint32_t *out_ids, float *out_dists,
                                       const uint32_t *nq_dev, etale_search_graph **out) {
    if (!idx || !out) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    *out = nullptr;
    const u32 L = beam > k ? beam : k;
    if (nq_max == 0 || k == 0 || L > 256 || !nq_dev)
        return idx->fail(ETALE_EINVAL, "graph needs nq_max > 0, k > 0, beam <= 256 and nq_dev");
    if (!is_device_ptr(queries) || !is_device_ptr(out_ids) || !is_device_ptr(out_dists) || !is_device_ptr(nq_dev))
        return idx->fail(ETALE_EINVAL, "graph buffers must be device pointers");
    if (idx->search_prec && k > 64) return idx->fail(ETALE_EINVAL, "reduced-precision search needs k <= 64");
    etale_search_graph *g = new etale_search_graph();
    g->idx = idx;
    if (cudaMalloc(&g->qpad, (size_t)nq_max * idx->mp * 4) != cudaSuccess ||
        cudaMalloc(&g->seed, (size_t)nq_max * L * 8) != cudaSuccess) {
        cudaGetLastError();
        etale_search_graph_destroy(g);
        return idx->fail(ETALE_ENOMEM, "graph scratch");
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        etale_search_graph_destroy(g);
        return idx->fail(ETALE_ECUDA, "capture stream");
    }
    const Dev d = idx->dev();
    const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * L;
    // Seeds on tensor cores (the batch size read on the device) when the
    // entry set is full, so that its size cannot change under the graph, and
    // writers do not run concurrently; else the CUDA-core seed kernel.
    const u32 S = idx->n_entries;
    SeedTcPlan tp{};
    SeedTcBufs tb{};
    if (idx->search_prec == 0 && idx->seed_tc && !idx->concurrent && S > 0 && S == idx->cfg.n_entry &&
        nq_max >= 32) {
        tp = seed_tc_plan(idx->dim, S, nq_max);
        if (idx->sd_E.p && cudaMalloc(&g->tA, tp.bytes_A) == cudaSuccess &&
            cudaMalloc(&g->tqstat, (size_t)nq_max * 16) == cudaSuccess &&
            cudaMalloc(&g->tkeys, tp.bytes_keys) == cudaSuccess &&
            cudaMalloc(&g->tfb, (size_t)nq_max * 4) == cudaSuccess && cudaMalloc(&g->tctr, 64) == cudaSuccess) {
            g->tc = true;
            g->S = S;
            g->launches = 6;
            tb = idx->seed_bufs();
            tb.A = g->tA;
            tb.qstat = g->tqstat;
            tb.keys = g->tkeys;
            tb.fb = g->tfb;
            tb.ctr = g->tctr;
            for (DevBuf *p : {&idx->sd_E, &idx->sd_en, &idx->sd_estat}) p->pins++;
            idx->round_graphs++;
        } else {
            cudaGetLastError();
        }
    }
    auto enqueue = [&]() {
        cudaError_t e = launch_ingest(g->qpad, idx->mp, queries, idx->dim, nq_max, cs, nq_dev);
        if (e == cudaSuccess)
            e = g->tc ? launch_seed_tc(d, g->qpad, nq_max, S, L, g->seed, tp, tb, idx->num_sms, cs, nq_dev)
                      : launch_seed(d, g->qpad, nq_max, L, g->seed, cs, idx->search_prec, nq_dev);
        if (e == cudaSuccess)
            e = launch_search(d, g->qpad, nq_max, L, H, 0, k, out_ids, out_dists, nullptr, nullptr, g->seed,
                              fit_tuning(idx, L, idx->tune), idx->num_sms, cs, idx->search_prec, idx->cfg.rerank, nq_dev);
        return e;
    };
    // one eager run sets the kernels' attributes outside the capture
    cudaError_t e = enqueue();
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t e2 = enqueue();
        e = cudaStreamEndCapture(cs, &g->graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        etale_search_graph_destroy(g);
        return idx->cuda_fail(e, "graph capture");
    }
    *out = g;
    return ETALE_OK;
}

etale_status etale_search_graph_launch(etale_search_graph *g, void *stream) {
    if (!g) return ETALE_EINVAL;
    if (g->tc && (g->idx->n_entries != g->S || g->idx->concurrent))
        return g->idx->fail(ETALE_EINVAL, "graph recorded with tensor-core seeding: the entry set must keep its "
                                          "size and writers must not run concurrently");
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return g->idx->cuda_fail(e, "graph launch");
    g_kernel_launches += g->launches;
    if (g->idx->concurrent) {
        std::lock_guard<std::mutex> lk(g->idx->mu);
        CK2(g->idx, cudaEventRecord(g->idx->search_ev, (cudaStream_t)stream), "record search event");
        g->idx->search_ev_valid = true;
    }
    return ETALE_OK;
}

etale_status etale_search_graph_check(etale_search_graph *g, void *stream) {
    if (!g) return ETALE_EINVAL;
    return check_search_errors(g->idx, (cudaStream_t)stream);
}

etale_status etale_search_graph_destroy(etale_search_graph *g) {
    if (!g) return ETALE_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaFree(g->qpad);
    cudaFree(g->seed);
    if (g->tc) {
        for (DevBuf *p : {&g->idx->sd_E, &g->idx->sd_en, &g->idx->sd_estat}) p->pins--;
        g->idx->round_graphs--;
    }
    cudaFree(g->tA);
    cudaFree(g->tqstat);
    cudaFree(g->tkeys);
    cudaFree(g->tfb);
    cudaFree(g->tctr);
    delete g;
    return ETALE_OK;
}

// ---------------------------------------------------------------------------
// Round graphs: one churn round (delete with repair, insert with refine,
// reclaim, and optionally a query batch) recorded once as a CUDA graph and
// replayed with one launch.  Sizes that change from round to round (next_id,
// the first new id, the live count, |E|) are read by the kernels from the
// index's device round state; the host never reads or waits in between.
// ---------------------------------------------------------------------------
struct etale_round_graph {
    etale_index *idx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    u32 n_del = 0, n_ins = 0, nq = 0, k = 0, L = 0;
    const u32 *del_ids = nullptr;
    const float *ins = nullptr, *queries = nullptr;
    u32 *out_ids = nullptr;
    float *out_dists = nullptr;
    float *ins_q = nullptr, *q_pad = nullptr;   // padded rows, fixed addresses
    u64 *q_seed = nullptr;
    bool seed_tc = false;
    u64 kernels = 0;                             // kernel nodes per replay
    u64 live_lb = 0;                             // host lower bound of the live count
    std::vector<DevBuf *> pinned;
};

namespace {

// Entry set from the device's live count (a recorded round).
cudaError_t rg_entries(etale_index *idx, etale_round_graph *g, const Dev &dg, cudaStream_t st) {
    const u64 cap = idx->capacity;
    ScanScratch ss;
    scan_scratch_carve(ss, as<u32>(idx->live_scan_scr), (u32)cap);
    cudaError_t e = launch_live_flags(dg, cap, as<u32>(idx->live_flags), st);
    if (e == cudaSuccess) e = exclusive_scan(as<u32>(idx->live_flags), as<u32>(idx->live_rank), (u32)cap, ss, st);
    if (e == cudaSuccess)
        e = launch_entries_select(dg, cap, as<u32>(idx->live_flags), as<u32>(idx->live_rank), 0, idx->cfg.n_entry, st);
    if (e == cudaSuccess && g->seed_tc) {
        const SeedTcPlan p = seed_tc_plan(idx->dim, idx->cfg.n_entry, 0);
        e = launch_seed_tc_entries(dg, idx->cfg.n_entry, p, idx->seed_bufs(), st);
    }
    return e;
}

cudaError_t rg_seed(etale_index *idx, etale_round_graph *g, const Dev &dg, const float *q, u32 nq, u32 L, u64 *seed,
                    cudaStream_t st, u32 prec = 0) {
    if (prec) return launch_seed(dg, q, nq, L, seed, st, prec);
    if (g->seed_tc && nq >= 32) {
        const SeedTcPlan p = seed_tc_plan(idx->dim, idx->cfg.n_entry, nq);
        return launch_seed_tc(dg, q, nq, idx->cfg.n_entry, L, seed, p, idx->seed_bufs(), idx->num_sms, st);
    }
    return launch_seed(dg, q, nq, L, seed, st, 0);
}

cudaError_t rg_offers(etale_index *idx, const Dev &dg, u32 nslots, cudaStream_t st) {
    Offers of{as<u32>(idx->of_key), as<u32>(idx->of_val), as<u32>(idx->of_key2), as<u32>(idx->of_val2),
              as<u32>(idx->of_src), as<float>(idx->of_rho), nslots};
    u64 *seg_count = as<u64>(idx->counts) + 0;
    cudaError_t e = cudaSuccess;
    if (idx->cfg.mode == ETALE_MODE_LOCKFREE) {
        e = launch_offer_fold(dg, of, nullptr, seg_count, idx->cfg.cas_budget, idx->num_sms, st, 0, nslots);
    } else {
        SortScratch ss;
        sort_scratch_carve(ss, as<u32>(idx->sort_scr), nslots);
        ScanScratch sc;
        scan_scratch_carve(sc, as<u32>(idx->scan_scr), nslots);
        e = radix_sort_pairs(of.key, of.val, of.key_alt, of.val_alt, nslots, bits_for(idx->capacity), ss, st);
        if (e == cudaSuccess)
            e = make_segments(of.key, nslots, (u32)idx->capacity, as<u32>(idx->seg_flags), as<u32>(idx->seg_scan),
                              as<u32>(idx->seg_start), seg_count, sc, st);
        if (e == cudaSuccess)
            e = launch_offer_fold(dg, of, as<u32>(idx->seg_start), seg_count, 0, idx->num_sms, st);
    }
    if (e == cudaSuccess) e = launch_recycle(dg, st);
    return e;
}

// The phase sequence of one round, as the eager calls run it for a delete
// batch of n_del ids (NIL entries are no-ops), one insert sub-batch of n_ins
// rows and a Reclaim, then the query batch.
cudaError_t rg_enqueue(etale_index *idx, etale_round_graph *g, cudaStream_t st) {
    Dev dg = idx->dev();
    dg.rs = idx->rs;
    const u32 R = idx->R;
    const u64 cap = idx->capacity;
    cudaError_t e = cudaSuccess;
    if (g->n_del) {
        const u32 n = g->n_del, slots = n * R;
        SortScratch ss;
        sort_scratch_carve(ss, as<u32>(idx->sort_scr), std::max(slots, n));
        ScanScratch sc;
        scan_scratch_carve(sc, as<u32>(idx->scan_scr), std::max(slots, n));
        u64 *n_dt = as<u64>(idx->counts) + 1, *seg_count = as<u64>(idx->counts) + 2;
        const u32 invalid = (u32)cap;
        e = cudaMemcpyAsync(idx->del_ids.p, g->del_ids, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = launch_fill_offer_keys(as<u32>(idx->del_vals2), as<u32>(idx->del_vals), n, 0, st);
        if (e == cudaSuccess)
            e = radix_sort_pairs(as<u32>(idx->del_ids), as<u32>(idx->del_vals), as<u32>(idx->del_ids2),
                                 as<u32>(idx->del_vals2), n, 32, ss, st);
        if (e == cudaSuccess) e = launch_tombstone(dg, as<u32>(idx->del_ids), n, cap, as<u32>(idx->del_ok), st);
        if (e == cudaSuccess) e = exclusive_scan(as<u32>(idx->del_ok), as<u32>(idx->del_scan), n, sc, st);
        if (e == cudaSuccess)
            e = launch_compact_ok(as<u32>(idx->del_ids), as<u32>(idx->del_ok), as<u32>(idx->del_scan), n,
                                  as<u32>(idx->dt), n_dt, st);
        if (e == cudaSuccess) e = launch_round_add(idx->rs, RS_DELETED, n_dt, st);
        if (e == cudaSuccess) e = launch_fill_offer_keys(as<u32>(idx->pair_key), as<u32>(idx->pair_val), slots, invalid, st);
        if (e == cudaSuccess)
            e = launch_repair_k(dg, as<u32>(idx->dt), n_dt, n, as<u32>(idx->pair_key), as<u32>(idx->pair_val),
                                as<uint2>(idx->pair_K), as<u32>(idx->pair_Kn), idx->num_sms, st);
        if (idx->cfg.mode == ETALE_MODE_LOCKFREE) {
            if (e == cudaSuccess)
                e = launch_repair_fold(dg, as<u32>(idx->dt), as<u32>(idx->pair_key), as<u32>(idx->pair_val),
                                       as<uint2>(idx->pair_K), as<u32>(idx->pair_Kn), nullptr, seg_count, slots,
                                       idx->cfg.cas_budget, idx->num_sms, st, 0);
        } else {
            if (e == cudaSuccess)
                e = radix_sort_pairs(as<u32>(idx->pair_key), as<u32>(idx->pair_val), as<u32>(idx->pair_key2),
                                     as<u32>(idx->pair_val2), slots, bits_for(cap), ss, st);
            if (e == cudaSuccess)
                e = make_segments(as<u32>(idx->pair_key), slots, invalid, as<u32>(idx->pair_flags),
                                  as<u32>(idx->pair_scan), as<u32>(idx->pair_seg), seg_count, sc, st);
            if (e == cudaSuccess)
                e = launch_repair_fold(dg, as<u32>(idx->dt), as<u32>(idx->pair_key), as<u32>(idx->pair_val),
                                       as<uint2>(idx->pair_K), as<u32>(idx->pair_Kn), as<u32>(idx->pair_seg),
                                       seg_count, slots, 0, idx->num_sms, st);
        }
        if (e == cudaSuccess) e = launch_recycle(dg, st);
    }
    if (g->n_ins && e == cudaSuccess) {
        const u32 b = g->n_ins, Lb = idx->cfg.build_beam;
        const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * Lb;
        Offers of{as<u32>(idx->of_key), as<u32>(idx->of_val), as<u32>(idx->of_key2), as<u32>(idx->of_val2),
                  as<u32>(idx->of_src), as<float>(idx->of_rho), b * R};
        e = launch_round_advance(idx->rs, b, st);
        if (e == cudaSuccess) e = launch_ingest(idx->x, idx->mp, g->ins, idx->dim, b, st, nullptr, idx->rs + RS_FIRST);
        if (e == cudaSuccess) e = launch_ingest(g->ins_q, idx->mp, g->ins, idx->dim, b, st);
        if (e == cudaSuccess) e = launch_ingest_copies(dg, 0, b, st);
        if (e == cudaSuccess) e = rg_seed(idx, g, dg, g->ins_q, b, Lb, as<u64>(idx->seed), st, idx->insert_prec);
        if (e == cudaSuccess)
            e = launch_search(dg, g->ins_q, b, Lb, H, 1, 0, nullptr, nullptr, as<u64>(idx->exp_keys),
                              as<u32>(idx->exp_count), as<u64>(idx->seed), fit_tuning(idx, Lb, idx->tune), idx->num_sms,
                              st, idx->insert_prec, 4, nullptr, false);
        if (e == cudaSuccess)
            e = launch_prune_insert(dg, 0, b, as<u64>(idx->exp_keys), as<u32>(idx->exp_count), H, idx->cfg.max_cand,
                                    as<u32>(idx->F_id), as<float>(idx->F_rho), as<u32>(idx->F_n), of, idx->num_sms, st,
                                    idx->insert_prec != 0);
        if (e == cudaSuccess) e = launch_recycle(dg, st);
        if (e == cudaSuccess) e = rg_offers(idx, dg, b * R, st);
        const u32 rmode = idx->cfg.refine == 1 ? 0 : idx->cfg.refine;
        if (rmode && e == cudaSuccess) {
            const size_t sb = refine_spill_bytes(dg, idx->cfg.max_cand, idx->num_sms);
            e = launch_refine(dg, 0, b, rmode, idx->cfg.max_cand, of, idx->num_sms, st,
                              static_cast<char *>(idx->refine_spill.p), sb);
            if (e == cudaSuccess) e = launch_recycle(dg, st);
            if (e == cudaSuccess) e = rg_offers(idx, dg, b * R, st);
        }
        if (e == cudaSuccess) e = rg_entries(idx, g, dg, st);
    }
    // Reclaim: entry set first, then compaction and phase 2
    if (e == cudaSuccess) e = rg_entries(idx, g, dg, st);
    if (e == cudaSuccess) e = launch_tomb_bits(dg, cap, as<u32>(idx->tomb_bits), st);
    if (e == cudaSuccess) e = launch_compact(dg, cap, as<u32>(idx->tomb_bits), st);
    if (e == cudaSuccess) e = launch_recycle(dg, st);
    if (e == cudaSuccess) e = launch_reclaim_tombstones(dg, cap, st);
    if (e == cudaSuccess) e = launch_recycle(dg, st);
    if (g->nq && e == cudaSuccess) {
        const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * g->L;
        e = launch_ingest(g->q_pad, idx->mp, g->queries, idx->dim, g->nq, st);
        if (e == cudaSuccess) e = rg_seed(idx, g, dg, g->q_pad, g->nq, g->L, g->q_seed, st, idx->search_prec);
        if (e == cudaSuccess)
            e = launch_search(dg, g->q_pad, g->nq, g->L, H, 0, g->k, g->out_ids, g->out_dists, nullptr, nullptr,
                              g->q_seed, fit_tuning(idx, g->L, idx->tune), idx->num_sms, st, idx->search_prec,
                              idx->cfg.rerank, nullptr, false);
    }
    return e;
}

// Conditions under which a replay equals the eager calls: one insert
// sub-batch (n_ins <= live, <= max_batch), an entry set at its full size
// when seeding on tensor cores, ids left, and a pool that covers the round.
etale_status rg_check(etale_index *idx, etale_round_graph *g) {
    const u64 live_ins = g->live_lb > g->n_del ? g->live_lb - g->n_del : 0;   // live when the insert runs
    if (g->n_ins && (live_ins < g->n_ins || g->n_ins > idx->cfg.max_batch))
        return idx->fail(ETALE_EINVAL, "round graph: the insert would not be one sub-batch (live may be %llu)",
                         (unsigned long long)live_ins);
    if (g->seed_tc && live_ins < idx->cfg.n_entry)
        return idx->fail(ETALE_EINVAL, "round graph: the live set may fall below n_entry; record a new graph");
    if (idx->next_id + g->n_ins > idx->capacity) return idx->fail(ETALE_ECAPACITY, "round graph: id budget exhausted");
    // at a call boundary every id holds at most one slab and nothing is
    // retired; a phase pops at most two slabs per publication it attempts
    // (lock-free retries are rare; the device flags an empty pool) and the
    // compaction at most one per live node
    const u64 nid = idx->next_id + g->n_ins;
    const u64 need = nid + std::max<u64>({2ull * g->n_del * idx->R, 2ull * g->n_ins * (idx->R + 1), nid});
    if (idx->pool < need)
        return idx->fail(ETALE_ENOMEM, "round graph: the slab pool may not cover a round");
    return ETALE_OK;
}

}  // namespace

etale_status etale_round_graph_create(etale_index *idx, uint32_t n_del, const uint32_t *del_ids, uint32_t n_ins,
                                      const float *ins_vecs, uint32_t nq, uint32_t k, uint32_t beam,
                                      const float *queries, uint32_t *out_ids, float *out_dists,
                                      etale_round_graph **out) {
    if (!idx || !out) return ETALE_EINVAL;
    *out = nullptr;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (idx->concurrent) return idx->fail(ETALE_EINVAL, "round graphs are not available in concurrent mode");
    if ((n_del && !is_device_ptr(del_ids)) || (n_ins && !is_device_ptr(ins_vecs)) ||
        (nq && (!is_device_ptr(queries) || !is_device_ptr(out_ids) || !is_device_ptr(out_dists))))
        return idx->fail(ETALE_EINVAL, "round graph buffers must be device pointers");
    const u32 L = beam > k ? beam : k;
    if (nq && (k == 0 || L > 256)) return idx->fail(ETALE_EINVAL, "round graph queries need k > 0 and beam <= 256");
    if (nq && idx->search_prec && k > 64) return idx->fail(ETALE_EINVAL, "reduced-precision search needs k <= 64");
    if ((u64)n_del * idx->R > 0x7FFFFFFFull || (u64)n_ins * idx->R > 0x7FFFFFFFull)
        return idx->fail(ETALE_EINVAL, "round graph batch too large");
    etale_round_graph *g = new etale_round_graph();
    g->idx = idx;
    g->n_del = n_del; g->n_ins = n_ins; g->nq = nq; g->k = k; g->L = L;
    g->del_ids = del_ids; g->ins = ins_vecs; g->queries = queries; g->out_ids = out_ids; g->out_dists = out_dists;
    g->live_lb = idx->live;
    g->seed_tc = idx->seed_tc && idx->live >= (u64)idx->cfg.n_entry + n_del;
    auto bail = [&](etale_status s) {
        etale_round_graph_destroy(g);
        return s;
    };
    etale_status s = rg_check(idx, g);
    if (s != ETALE_OK) return bail(s);
    // every buffer the recording names is sized now and then pinned
    const u32 R = idx->R, Lb = idx->cfg.build_beam;
    const u64 cap = idx->capacity, mx = std::max<u64>({(u64)n_ins, (u64)nq, 1});
    const u64 nslot = std::max<u64>({(u64)n_del * R, (u64)n_ins * R, (u64)n_del, 1});
    const SeedTcPlan pe = seed_tc_plan(idx->dim, idx->cfg.n_entry, 0), pq = seed_tc_plan(idx->dim, idx->cfg.n_entry, (u32)mx);
    Dev d0 = idx->dev();
    bool ok = size_delete_scratch(idx, std::max<u32>(n_del, 1)) && size_batch_scratch(idx, std::max<u32>(n_ins, 1)) == ETALE_OK &&
              grow(idx->sort_scr, sort_scratch_elems((u32)nslot) * 4) && grow(idx->scan_scr, scan_scratch_elems((u32)nslot) * 4) &&
              grow(idx->seed, (size_t)std::max<u32>(n_ins, 1) * Lb * 8) &&
              grow(idx->refine_spill, refine_spill_bytes(d0, idx->cfg.max_cand, idx->num_sms)) &&
              grow(idx->live_flags, cap * 4) && grow(idx->live_rank, cap * 4) &&
              grow(idx->live_scan_scr, scan_scratch_elems((u32)cap) * 4) && grow(idx->tomb_bits, ((cap + 31) / 32) * 4);
    if (ok && g->seed_tc)
        ok = grow(idx->sd_E, pe.bytes_E) && grow(idx->sd_en, (size_t)pe.s_pad * 4) && grow(idx->sd_estat, 64) &&
             grow(idx->sd_A, pq.bytes_A) && grow(idx->sd_qstat, (size_t)mx * 16) && grow(idx->sd_keys, pq.bytes_keys) &&
             grow(idx->sd_fb, (size_t)mx * 4) && grow(idx->sd_ctr, 64);
    if (!ok) return bail(idx->fail(ETALE_ENOMEM, "round graph scratch"));
    if ((n_ins && cudaMalloc(&g->ins_q, (size_t)n_ins * idx->mp * 4) != cudaSuccess) ||
        (nq && (cudaMalloc(&g->q_pad, (size_t)nq * idx->mp * 4) != cudaSuccess ||
                cudaMalloc(&g->q_seed, (size_t)nq * L * 8) != cudaSuccess))) {
        cudaGetLastError();
        return bail(idx->fail(ETALE_ENOMEM, "round graph buffers"));
    }
    // pin every index buffer the recording names
    DevBuf *pins[] = {&idx->del_ids, &idx->del_vals, &idx->del_ids2, &idx->del_vals2, &idx->del_ok, &idx->del_scan,
                      &idx->dt, &idx->pair_key, &idx->pair_val, &idx->pair_key2, &idx->pair_val2, &idx->pair_K,
                      &idx->pair_Kn, &idx->pair_flags, &idx->pair_scan, &idx->pair_seg, &idx->counts,
                      &idx->sort_scr, &idx->scan_scr, &idx->exp_keys, &idx->exp_count, &idx->F_id, &idx->F_rho,
                      &idx->F_n, &idx->of_key, &idx->of_val, &idx->of_key2, &idx->of_val2, &idx->of_src,
                      &idx->of_rho, &idx->seg_flags, &idx->seg_scan, &idx->seg_start, &idx->seed,
                      &idx->refine_spill, &idx->live_flags, &idx->live_rank, &idx->live_scan_scr, &idx->tomb_bits,
                      &idx->sd_E, &idx->sd_en, &idx->sd_estat, &idx->sd_A, &idx->sd_qstat, &idx->sd_keys,
                      &idx->sd_fb, &idx->sd_ctr};
    for (DevBuf *p : pins) {
        p->pins++;
        g->pinned.push_back(p);
    }
    idx->round_graphs++;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return bail(idx->fail(ETALE_ECUDA, "capture stream"));
    const bool prof = idx->prof;
    idx->prof = false;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t e2 = rg_enqueue(idx, g, cs);
        e = cudaStreamEndCapture(cs, &g->graph);
        if (e == cudaSuccess) e = e2;
    }
    idx->prof = prof;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e == cudaSuccess) {
        size_t nn = 0;
        e = cudaGraphGetNodes(g->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g->graph, nodes.data(), &nn);
        for (size_t i = 0; e == cudaSuccess && i < nn; i++) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) g->kernels++;
        }
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(idx->cuda_fail(e, "round graph capture"));
    }
    *out = g;
    return ETALE_OK;
}

etale_status etale_round_graph_launch(etale_round_graph *g, void *stream) {
    if (!g) return ETALE_EINVAL;
    etale_index *idx = g->idx;
    if (!idx->graph_pending) g->live_lb = idx->live;
    etale_status s = rg_check(idx, g);
    if (s != ETALE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_round_set(idx->rs, idx->next_id, st), "round state");
    CK(cudaGraphLaunch(g->exec, st), "round graph launch");
    CK(cudaEventRecord(idx->graph_ev, st), "round graph event");
    g_kernel_launches += g->kernels + 1;
    idx->next_id += g->n_ins;
    idx->graph_pending = true;
    g->live_lb = g->live_lb + g->n_ins - std::min<u64>(g->live_lb, g->n_del);
    return ETALE_OK;
}

etale_status etale_round_graph_sync(etale_round_graph *g) {
    if (!g) return ETALE_EINVAL;
    etale_status s = settle(g->idx);
    g->live_lb = g->idx->live;
    return s;
}

etale_status etale_round_graph_destroy(etale_round_graph *g) {
    if (!g) return ETALE_OK;
    if (g->idx) {
        if (g->idx->graph_pending) settle(g->idx);
        for (DevBuf *p : g->pinned) p->pins--;
        if (!g->pinned.empty()) g->idx->round_graphs--;
    }
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaFree(g->ins_q);
    cudaFree(g->q_pad);
    cudaFree(g->q_seed);
    delete g;
    return ETALE_OK;
}

// ---------------------------------------------------------------------------
// Serving ring (see launch_ring_search): slots of query rows and results in
// pinned, mapped host memory, so that the host submits and collects without
// copies and a running launch sees new submissions.
// ---------------------------------------------------------------------------
struct etale_ring {
    etale_index *idx = nullptr;
    u32 slots = 0, k = 0, L = 0, seq = 0;
    void *host = nullptr;                 // one mapped allocation
    float *rows = nullptr;                // slots x mp
    u32 *ids = nullptr, *served_by = nullptr;
    float *dists = nullptr;
    u64 *done = nullptr, *ctl = nullptr;  // ctl[0] tail, ctl[1] closed
    float *d_rows = nullptr;
    u32 *d_ids = nullptr, *d_served = nullptr;
    float *d_dists = nullptr;
    u64 *d_done = nullptr, *d_ctl = nullptr;
    u64 *head = nullptr, *seed = nullptr; // device memory
    u64 tickets = 0;                      // tickets published so far (etale_ring_serve)
    cudaStream_t alt = nullptr;           // etale_ring_serve's second launch stream
};

etale_status etale_ring_create(etale_index *idx, uint32_t slots, uint32_t k, uint32_t beam, etale_ring **out) {
    if (!idx || !out) return ETALE_EINVAL;
    *out = nullptr;
    const u32 L = beam > k ? beam : k;
    if (slots == 0 || slots > (1u << 24) || k == 0 || L > 256)
        return idx->fail(ETALE_EINVAL, "ring needs 1..2^24 slots, k > 0 and beam <= 256");
    if (idx->search_prec && k > 64) return idx->fail(ETALE_EINVAL, "reduced-precision search needs k <= 64");
    etale_ring *r = new etale_ring();
    r->idx = idx; r->slots = slots; r->k = k; r->L = L;
    const size_t b_rows = (size_t)slots * idx->mp * 4, b_ids = (size_t)slots * k * 4, b_served = (size_t)slots * 4;
    const size_t o_ids = (b_rows + 255) / 256 * 256, o_dists = o_ids + (b_ids + 255) / 256 * 256;
    const size_t o_done = o_dists + (b_ids + 255) / 256 * 256, o_served = o_done + ((size_t)slots * 8 + 255) / 256 * 256;
    const size_t o_ctl = o_served + (b_served + 255) / 256 * 256, total = o_ctl + 256;
    char *d = nullptr;
    bool ok = cudaHostAlloc(&r->host, total, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&d, r->host, 0) == cudaSuccess &&
              cudaMalloc(&r->head, 64) == cudaSuccess && cudaMemset(r->head, 0, 64) == cudaSuccess &&
              cudaMalloc(&r->seed, (size_t)slots * L * 8) == cudaSuccess &&
              cudaStreamCreateWithFlags(&r->alt, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        etale_ring_destroy(r);
        return idx->fail(ETALE_ENOMEM, "ring allocation");
    }
    memset(r->host, 0, total);
    char *h = static_cast<char *>(r->host);
    r->rows = reinterpret_cast<float *>(h); r->d_rows = reinterpret_cast<float *>(d);
    r->ids = reinterpret_cast<u32 *>(h + o_ids); r->d_ids = reinterpret_cast<u32 *>(d + o_ids);
    r->dists = reinterpret_cast<float *>(h + o_dists); r->d_dists = reinterpret_cast<float *>(d + o_dists);
    r->done = reinterpret_cast<u64 *>(h + o_done); r->d_done = reinterpret_cast<u64 *>(d + o_done);
    r->served_by = reinterpret_cast<u32 *>(h + o_served); r->d_served = reinterpret_cast<u32 *>(d + o_served);
    r->ctl = reinterpret_cast<u64 *>(h + o_ctl); r->d_ctl = reinterpret_cast<u64 *>(d + o_ctl);
    *out = r;
    return ETALE_OK;
}

etale_status etale_ring_buffers(etale_ring *r, float **rows, uint32_t *row_stride, uint32_t **ids, float **dists,
                                uint64_t **done, uint32_t **served_by) {
    if (!r) return ETALE_EINVAL;
    if (rows) *rows = r->rows;
    if (row_stride) *row_stride = r->idx->mp;
    if (ids) *ids = r->ids;
    if (dists) *dists = r->dists;
    if (done) *done = reinterpret_cast<uint64_t *>(r->done);
    if (served_by) *served_by = r->served_by;
    return ETALE_OK;
}

etale_status etale_ring_publish(etale_ring *r, uint64_t tail) {
    if (!r) return ETALE_EINVAL;
    __atomic_store_n(&r->ctl[0], tail, __ATOMIC_RELEASE);
    return ETALE_OK;
}

etale_status etale_ring_close(etale_ring *r, int closed) {
    if (!r) return ETALE_EINVAL;
    __atomic_store_n(&r->ctl[1], (u64)(closed != 0), __ATOMIC_RELEASE);
    return ETALE_OK;
}

etale_status etale_ring_launch(etale_ring *r, uint32_t max_us, uint32_t blocks, uint32_t *seq, void *stream) {
    if (!r) return ETALE_EINVAL;
    etale_index *idx = r->idx;
    if (max_us == 0 || max_us > 1000000) return idx->fail(ETALE_EINVAL, "max_us must be 1..1e6");
    if (blocks == 0) blocks = (u32)idx->num_sms;   // two launches overlap in etale_ring_serve
    cudaStream_t st = (cudaStream_t)stream;
    const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * r->L;
    Dev d = idx->dev();
    const u32 sq = ++r->seq;
    CK(launch_ring_search(d, r->d_rows, r->slots, r->L, H, r->k, r->d_ids, r->d_dists, r->seed,
                          fit_tuning(idx, r->L, idx->tune), blocks, st, idx->search_prec, idx->cfg.rerank, r->head,
                          r->d_ctl, r->d_ctl + 1, r->d_done, r->d_served, sq, (u64)max_us * 1000ull),
       "ring launch");
    g_kernel_launches++;
    if (seq) *seq = sq;
    if (idx->concurrent) {
        std::lock_guard<std::mutex> lk(idx->mu);
        if (st == r->alt) {
            CK(cudaEventRecord(idx->search_ev2, st), "record search event");
            idx->search_ev2_valid = true;
        } else {
            CK(cudaEventRecord(idx->search_ev, st), "record search event");
            idx->search_ev_valid = true;
        }
    }
    return ETALE_OK;
}

etale_status etale_ring_stats(etale_ring *r, uint64_t *served, uint64_t *seed_ns, uint64_t *search_ns) {
    if (!r) return ETALE_EINVAL;
    u64 v[3];
    CK2(r->idx, cudaMemcpy(v, r->head + 4, sizeof(v), cudaMemcpyDeviceToHost), "ring statistics");
    if (served) *served = v[0];
    if (seed_ns) *seed_ns = v[1];
    if (search_ns) *search_ns = v[2];
    return ETALE_OK;
}

etale_status etale_ring_serve(etale_ring *r, const float *queries, const double *arrival_s, uint64_t n,
                             uint32_t max_us, uint32_t blocks, double *issued_s, double *completion_s,
                             uint32_t *out_ids, float *out_dists, uint64_t *mid_launch, uint32_t *launches,
                             void *stream) {
    if (!r || (n && (!queries || !arrival_s || !completion_s))) return ETALE_EINVAL;
    etale_index *idx = r->idx;
    if (max_us == 0 || max_us > 1000000) return idx->fail(ETALE_EINVAL, "max_us must be 1..1e6");
    for (u64 i = 1; i < n; i++)
        if (arrival_s[i] < arrival_s[i - 1]) return idx->fail(ETALE_EINVAL, "arrivals must ascend");
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    auto now_s = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    const u64 base = r->tickets, S = r->slots, K = r->k, dim = idx->dim, mp = idx->mp;
    std::vector<std::atomic<unsigned char>> collected(n);
    for (auto &c : collected) c.store(0);
    std::vector<double> issue_of_seq;         // host issue time of each launch of this call
    std::mutex seq_mu;
    std::atomic<bool> finished{false};
    std::atomic<u64> mids{0};
    std::atomic<u32> nlaunch{0};
    std::atomic<int> launch_err{0};
    const u32 seq0 = r->seq + 1;
    std::vector<double> issued_local(issued_s ? 0 : n);
    double *iss = issued_s ? issued_s : issued_local.data();
    __atomic_store_n(&r->ctl[1], 0ull, __ATOMIC_RELEASE);
    // Bounded launches, alternating between `stream` and the ring's second
    // stream: the next launch is issued when the current one has run three
    // quarters of its lifetime, so one launch is always taking tickets while
    // the one before it finishes the queries it holds.
    std::thread launcher([&]() {
        cudaStream_t sts[2] = {(cudaStream_t)stream, r->alt};
        for (u32 k = 0; !finished.load(); k++) {
            cudaStream_t s = sts[k & 1];
            uint32_t sq = 0;
            // the launch before last on this stream is past its lifetime
            if (cudaStreamSynchronize(s) != cudaSuccess) {
                launch_err.store(1);
                break;
            }
            if (finished.load()) break;
            {
                std::lock_guard<std::mutex> lk(seq_mu);
                issue_of_seq.push_back(now_s());
            }
            if (etale_ring_launch(r, max_us, blocks, &sq, s) != ETALE_OK) {
                launch_err.store(1);
                break;
            }
            nlaunch++;
            const double t_next = now_s() + 0.75e-6 * max_us;
            for (double t = now_s(); !finished.load() && t < t_next; t = now_s())
                std::this_thread::sleep_for(std::chrono::duration<double>(std::min(t_next - t, 200e-6)));
        }
        for (cudaStream_t s : sts)
            if (cudaStreamSynchronize(s) != cudaSuccess) launch_err.store(1);
    });
    // completions, in any order; results copied out before a slot is reused
    std::thread collector([&]() {
        u64 nxt = 0;
        std::vector<unsigned char> seen(n, 0);
        while (nxt < n && !launch_err.load()) {
            bool any = false;
            const u64 hi = std::min<u64>(n, nxt + S);
            for (u64 i = nxt; i < hi; i++) {
                if (seen[i]) continue;
                const u64 t = base + i, slot = t % S;
                if (__atomic_load_n(&r->done[slot], __ATOMIC_ACQUIRE) != t + 1) continue;
                completion_s[i] = now_s();
                if (out_ids) memcpy(out_ids + i * K, r->ids + slot * K, K * 4);
                if (out_dists) memcpy(out_dists + i * K, r->dists + slot * K, K * 4);
                const u32 sq = __atomic_load_n(&r->served_by[slot], __ATOMIC_RELAXED);
                {
                    std::lock_guard<std::mutex> lk(seq_mu);
                    if (sq >= seq0 && sq - seq0 < issue_of_seq.size() && issue_of_seq[sq - seq0] < iss[i]) mids++;
                }
                seen[i] = 1;
                collected[i].store(1, std::memory_order_release);
                any = true;
            }
            while (nxt < n && seen[nxt]) nxt++;
            if (!any) std::this_thread::sleep_for(std::chrono::microseconds(10));
        }
    });
    // submissions at their arrival times; a slot is rewritten only after its
    // previous query's results were collected
    u64 i = 0;
    while (i < n && !launch_err.load()) {
        const double now = now_s();
        if (arrival_s[i] > now) {
            const double wait = arrival_s[i] - now;
            if (wait > 50e-6) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait - 20e-6, 1e-3)));
            continue;
        }
        u64 j = i;
        while (j < n && arrival_s[j] <= now) {
            if (j >= S && !collected[j - S].load(std::memory_order_acquire)) break;
            const u64 slot = (base + j) % S;
            memcpy(r->rows + slot * mp, queries + j * dim, dim * 4);
            iss[j] = now_s();
            j++;
        }
        if (j > i) {
            __atomic_store_n(&r->ctl[0], base + j, __ATOMIC_RELEASE);
            i = j;
        } else {
            std::this_thread::sleep_for(std::chrono::microseconds(10));
        }
    }
    collector.join();
    finished.store(true);
    __atomic_store_n(&r->ctl[1], 1ull, __ATOMIC_RELEASE);   // the launch in flight ends now
    launcher.join();
    __atomic_store_n(&r->ctl[1], 0ull, __ATOMIC_RELEASE);
    r->tickets = base + n;
    if (mid_launch) *mid_launch = mids.load();
    if (launches) *launches = nlaunch.load();
    if (launch_err.load()) return idx->fail(ETALE_ECUDA, "ring launch failed during serving");
    return check_search_errors(idx, (cudaStream_t)stream);
}

etale_status etale_ring_destroy(etale_ring *r) {
    if (!r) return ETALE_OK;
    if (r->alt) {
        cudaStreamSynchronize(r->alt);
        cudaStreamDestroy(r->alt);
    }
    if (r->host) cudaFreeHost(r->host);
    cudaFree(r->head);
    cudaFree(r->seed);
    delete r;
    return ETALE_OK;
}

etale_status etale_ground_truth_info(etale_index *idx, uint32_t *path, uint64_t *fallback_queries) {
    if (!idx) return ETALE_EINVAL;
    if (path) *path = idx->gt_path;
    if (fallback_queries) *fallback_queries = idx->gt_fallbacks;
    return ETALE_OK;
}

etale_status etale_selftest_bounded_wait(uint32_t poll_limit, void *stream) {
    if (poll_limit < 1 || poll_limit > 1000000) {
        t_last_error = "poll_limit must be 1..1e6";
        return ETALE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    u32 *status = nullptr, h = 0;
    cudaError_t e = cudaMalloc(&status, 4);
    if (e == cudaSuccess) e = launch_selftest_wait(poll_limit, status, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (status) cudaFree(status);
    if (e != cudaSuccess) {
        t_last_error = std::string("selftest: ") + cudaGetErrorString(e);
        return ETALE_ECUDA;
    }
    g_kernel_launches++;
    if (h & ERR_TIMEOUT) {
        t_last_error = "a bounded device wait gave up (self-test)";
        return ETALE_ETIMEOUT;
    }
    return ETALE_OK;
}

etale_status etale_set_concurrent(etale_index *idx, int on) {
    if (!idx) return ETALE_EINVAL;
    idx->concurrent = on != 0;
    return ETALE_OK;
}

uint64_t etale_kernel_launches(const etale_index *) { return g_kernel_launches.load(); }

// ---------------------------------------------------------------------------
// etale_search_static: the query search with its scratch in a fixed
// file-scope device array instead of on-demand allocations.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[ETALE_STATIC_SCRATCH_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
void *g_static_scratch_ptr[MAX_DEVICES] = {};
std::mutex g_static_mu;

// Device address of g_static_scratch on the current device (looked up once
// per device; the host-side symbol is only a stand-in and must not be passed
// to a kernel).
cudaError_t static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_scratch_ptr[dev] = p;
    }
    *out = g_static_scratch_ptr[dev];
    return cudaSuccess;
}
}  // namespace

etale_status etale_search_static(etale_index *idx, const float *queries, uint64_t nq, uint32_t k, uint32_t beam,
                                 uint32_t *out_ids, float *out_dists, void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (nq == 0) return ETALE_OK;
    if (!queries || !out_ids || !out_dists || k == 0) return idx->fail(ETALE_EINVAL, "null buffer or k == 0");
    if (!is_device_ptr(queries) || !is_device_ptr(out_ids) || !is_device_ptr(out_dists))
        return idx->fail(ETALE_EINVAL, "etale_search_static takes device pointers only");
    const u32 L = beam > k ? beam : k;
    if (L > 256) return idx->fail(ETALE_EINVAL, "beam must be <= 256");
    if (idx->search_prec && k > 64) return idx->fail(ETALE_EINVAL, "reduced-precision search needs k <= 64");
    // Bound nq by a division first, so that the byte count below cannot wrap
    // (each query needs at least 4 * mp + 8 * L >= 12 bytes).
    const u64 per_query = 4ull * idx->mp + 8ull * L;
    if (nq > (u64)ETALE_STATIC_SCRATCH_BYTES / per_query)
        return idx->fail(ETALE_EINVAL, "etale_search_static: %llu queries need %llu bytes of scratch each, above the %u-byte limit",
                         (unsigned long long)nq, (unsigned long long)per_query, (unsigned)ETALE_STATIC_SCRATCH_BYTES);
    const size_t qbytes = ((size_t)nq * idx->mp * 4 + 255) / 256 * 256;
    const size_t need = qbytes + (size_t)nq * L * 8;
    if (need > ETALE_STATIC_SCRATCH_BYTES)
        return idx->fail(ETALE_EINVAL, "etale_search_static: %llu queries need %zu bytes of scratch, above the %u-byte limit",
                         (unsigned long long)nq, need, (unsigned)ETALE_STATIC_SCRATCH_BYTES);
    void *scr = nullptr;
    CK(static_scratch(&scr), "static scratch set-up");
    float *qpad = reinterpret_cast<float *>(scr);
    u64 *seed = reinterpret_cast<u64 *>(reinterpret_cast<unsigned char *>(scr) + qbytes);
    cudaStream_t st = (cudaStream_t)stream;
    Dev d = idx->dev();
    // every scratch byte read below is written first in this call (padded
    // rows by ingest, all L seed slots per query by the seed kernel)
    CK(launch_ingest(qpad, idx->mp, queries, idx->dim, nq, st), "query ingest");
    CK(launch_seed(d, qpad, (u32)nq, L, seed, st, idx->search_prec), "query seed");
    const u32 H = idx->cfg.max_hops ? idx->cfg.max_hops : 4 * L;
    CK(launch_search(d, qpad, (u32)nq, L, H, 0, k, out_ids, out_dists, nullptr, nullptr, seed, fit_tuning(idx, L, idx->tune),
                     idx->num_sms, st, idx->search_prec, idx->cfg.rerank),
       "search");
    g_kernel_launches += 3;
    if (idx->concurrent) {
        std::lock_guard<std::mutex> lk(idx->mu);
        CK(cudaEventRecord(idx->search_ev, st), "record search event");
        idx->search_ev_valid = true;
    }
    return check_search_errors(idx, st);
}

// ---------------------------------------------------------------------------
// Snapshots (format in include/etale.h).  Chunked by ids so that host memory
// stays bounded at 10M-row indexes.
// ---------------------------------------------------------------------------
namespace {
constexpr char SNAP_MAGIC[8] = {'E', 'T', 'A', 'L', 'E', 'S', 'N', '1'};
constexpr u32 SNAP_NCFG = 17;
constexpr u64 SNAP_CHUNK = 1ull << 18;

void cfg_to_words(const etale_config &c, u64 *w) {
    u32 ab;
    memcpy(&ab, &c.alpha, 4);
    const u64 v[SNAP_NCFG] = {c.build_beam, ab, c.max_hops, c.max_cand, c.refine, c.max_batch, c.pool_slabs,
                              c.n_entry, c.mode, c.cas_budget, c.stage_kb, c.gram, c.copies, c.rerank,
                              c.gt, c.seed, c.exact_rows};
    memcpy(w, v, sizeof v);
}
void words_to_cfg(const u64 *w, etale_config &c) {
    memset(&c, 0, sizeof c);
    u32 ab = (u32)w[1];
    c.build_beam = (u32)w[0]; memcpy(&c.alpha, &ab, 4); c.max_hops = (u32)w[2]; c.max_cand = (u32)w[3];
    c.refine = (u32)w[4]; c.max_batch = w[5]; c.pool_slabs = w[6]; c.n_entry = (u32)w[7]; c.mode = (u32)w[8];
    c.cas_budget = (u32)w[9]; c.stage_kb = (u32)w[10]; c.gram = (u32)w[11]; c.copies = (u32)w[12];
    c.rerank = (u32)w[13]; c.gt = (u32)w[14]; c.seed = (u32)w[15]; c.exact_rows = (u32)w[16];
}

struct File {
    FILE *f = nullptr;
    ~File() { if (f) fclose(f); }
};
}  // namespace

etale_status etale_save(etale_index *idx, const char *path, void *stream) {
    if (!idx) return ETALE_EINVAL;
    {
        etale_status s_ = settle(idx);
        if (s_ != ETALE_OK) return s_;
    }
    if (!path) return idx->fail(ETALE_EINVAL, "path is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st), "synchronize");
    File f;
    f.f = fopen(path, "wb");
    if (!f.f) return idx->fail(ETALE_EINVAL, "cannot open %s for writing", path);
    const u64 n = idx->next_id, R = idx->R;
    const u32 ne = idx->n_entries;
    bool ok = fwrite(SNAP_MAGIC, 1, 8, f.f) == 8;
    const u32 h32[4] = {1u, idx->dim, idx->metric, idx->R};
    const u64 h64[2] = {idx->capacity, n};
    const u32 h32b[2] = {ne, SNAP_NCFG};
    u64 cw[SNAP_NCFG];
    cfg_to_words(idx->cfg, cw);
    ok = ok && fwrite(h32, 4, 4, f.f) == 4 && fwrite(h64, 8, 2, f.f) == 2 && fwrite(h32b, 4, 2, f.f) == 2 &&
         fwrite(cw, 8, SNAP_NCFG, f.f) == SNAP_NCFG;
    // vectors, unpadded
    std::vector<float> xh;
    for (u64 lo = 0; lo < n && ok; lo += SNAP_CHUNK) {
        const u64 c = std::min(SNAP_CHUNK, n - lo);
        xh.resize(c * idx->dim);
        CK(cudaMemcpy2D(xh.data(), (size_t)idx->dim * 4, idx->x + lo * idx->mp, (size_t)idx->mp * 4,
                        (size_t)idx->dim * 4, c, cudaMemcpyDeviceToHost),
           "save vectors");
        ok = fwrite(xh.data(), 4, c * idx->dim, f.f) == c * idx->dim;
    }
    // flags and degrees from the reference words; lists from the export kernel
    std::vector<u64> refh(n);
    if (n) CK(cudaMemcpy(refh.data(), idx->ref, n * 8, cudaMemcpyDeviceToHost), "save references");
    std::vector<unsigned char> fl(n), dg(n);
    for (u64 u = 0; u < n; u++) {
        const u64 r = refh[u];
        const bool hs = ref_slab(r) != NIL;
        fl[u] = (unsigned char)(ref_del(r) | (hs ? 2u : 0u) | (hs && ref_pruned(r) ? 4u : 0u));
        dg[u] = hs ? (unsigned char)ref_deg(r) : 0;
    }
    ok = ok && fwrite(fl.data(), 1, n, f.f) == n && fwrite(dg.data(), 1, n, f.f) == n;
    if (n && ok) {
        const u64 c0 = std::min(SNAP_CHUNK, n);
        if (!grow(idx->ex_del, c0) || !grow(idx->ex_hs, c0) || !grow(idx->ex_deg, c0) ||
            !grow(idx->ex_ids, c0 * R * 4) || !grow(idx->ex_rho, c0 * R * 4))
            return idx->fail(ETALE_ENOMEM, "save staging");
        std::vector<u32> ids(c0 * R);
        std::vector<float> rho(c0 * R);
        std::vector<uint2> out;
        for (u64 lo = 0; lo < n && ok; lo += SNAP_CHUNK) {
            const u64 c = std::min(SNAP_CHUNK, n - lo);
            Dev d = idx->dev();
            d.ref = idx->ref + lo;   // the export kernel reads ids [0, c) of this view
            CK(launch_export(d, c, as<unsigned char>(idx->ex_del), as<unsigned char>(idx->ex_hs),
                             as<unsigned char>(idx->ex_deg), as<u32>(idx->ex_ids), as<float>(idx->ex_rho), st),
               "save export");
            g_kernel_launches++;
            CK(cudaMemcpyAsync(ids.data(), idx->ex_ids.p, c * R * 4, cudaMemcpyDeviceToHost, st), "save lists");
            CK(cudaMemcpyAsync(rho.data(), idx->ex_rho.p, c * R * 4, cudaMemcpyDeviceToHost, st), "save lists");
            CK(cudaStreamSynchronize(st), "synchronize");
            out.clear();
            for (u64 i = 0; i < c; i++)
                for (u32 j = 0; j < dg[lo + i]; j++) {
                    uint2 e;
                    e.x = ids[i * R + j];
                    memcpy(&e.y, &rho[i * R + j], 4);
                    out.push_back(e);
                }
            ok = fwrite(out.data(), 8, out.size(), f.f) == out.size();
        }
    }
    if (ne && ok) {
        std::vector<u32> eh(ne);
        CK(cudaMemcpy(eh.data(), idx->entries, (size_t)ne * 4, cudaMemcpyDeviceToHost), "save entries");
        ok = fwrite(eh.data(), 4, ne, f.f) == ne;
    }
    ok = ok && fflush(f.f) == 0;
    if (!ok) return idx->fail(ETALE_EINVAL, "write to %s failed", path);
    return ETALE_OK;
}

etale_status etale_load(const char *path, const etale_config *cfg_in, uint64_t capacity, etale_index **out) {
    if (!out) { t_last_error = "out is NULL"; return ETALE_EINVAL; }
    *out = nullptr;
    auto bad = [](const char *m) { t_last_error = m; return ETALE_EINVAL; };
    if (!path) return bad("path is NULL");
    File f;
    f.f = fopen(path, "rb");
    if (!f.f) return bad("cannot open the snapshot file");
    char magic[8];
    u32 h32[4], h32b[2];
    u64 h64[2], cw[SNAP_NCFG];
    if (fread(magic, 1, 8, f.f) != 8 || memcmp(magic, SNAP_MAGIC, 8) != 0) return bad("not an ETALE snapshot (magic)");
    if (fread(h32, 4, 4, f.f) != 4 || h32[0] != 1u) return bad("unsupported snapshot version");
    if (fread(h64, 8, 2, f.f) != 2 || fread(h32b, 4, 2, f.f) != 2 || h32b[1] != SNAP_NCFG ||
        fread(cw, 8, SNAP_NCFG, f.f) != SNAP_NCFG)
        return bad("truncated snapshot header");
    const u32 dim = h32[1], metric = h32[2], R = h32[3];
    const u64 n = h64[1];
    const u32 ne = h32b[0];
    if (capacity == 0) capacity = h64[0];
    if (n > capacity) return bad("capacity below the saved next_id");
    etale_config cfg;
    if (cfg_in) cfg = *cfg_in;
    else words_to_cfg(cw, cfg);
    etale_index *idx = nullptr;
    etale_status s = etale_create(dim, (etale_metric)metric, R, capacity, &cfg, &idx);
    if (s != ETALE_OK) return s;
    auto fail = [&](etale_status e, const char *m) {
        t_last_error = m;
        etale_destroy(idx);
        return e;
    };
    if (ne > idx->cfg.n_entry) return fail(ETALE_EINVAL, "saved entry set larger than n_entry");
    std::vector<float> xh;
    for (u64 lo = 0; lo < n; lo += SNAP_CHUNK) {
        const u64 c = std::min(SNAP_CHUNK, n - lo);
        xh.resize(c * dim);
        if (fread(xh.data(), 4, c * dim, f.f) != c * dim) return fail(ETALE_EINVAL, "truncated vectors");
        if (cudaMemcpy2D(idx->x + lo * idx->mp, (size_t)idx->mp * 4, xh.data(), (size_t)dim * 4, (size_t)dim * 4, c,
                         cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(ETALE_ECUDA, "load vectors");
    }
    std::vector<unsigned char> fl(n), dg(n);
    if (fread(fl.data(), 1, n, f.f) != n || fread(dg.data(), 1, n, f.f) != n) return fail(ETALE_EINVAL, "truncated flags");
    u64 used = 0, live = 0, tombs = 0, reclaimed = 0;
    for (u64 u = 0; u < n; u++) {
        const bool del = fl[u] & 1u, hs = (fl[u] >> 1) & 1u;
        if (fl[u] > 7u || dg[u] > R || (!hs && dg[u] != 0)) return fail(ETALE_EINVAL, "inconsistent flags or degree");
        used += hs;
        if (hs && !del) live++;
        else if (hs) tombs++;
        else if (del) reclaimed++;
    }
    if (used > idx->pool) return fail(ETALE_ENOMEM, "slab pool smaller than the saved lists");
    // slabs in ascending id order: the k-th id with a slab gets slab k; the free
    // stack as etale_create laid it out (slab P - 1 - i at position i) then holds
    // exactly the slabs >= used below its top
    std::vector<u64> refh(n);
    std::vector<uint2> slabh;
    u64 k = 0, kflush = 0;
    for (u64 u = 0; u < n; u++) {
        const bool del = fl[u] & 1u, hs = (fl[u] >> 1) & 1u;
        if (!hs) { refh[u] = ref_pack(del, 0, NIL); continue; }
        const size_t at = slabh.size();
        slabh.resize(at + R, make_uint2(NIL, 0u));
        if (dg[u] && fread(slabh.data() + at, 8, dg[u], f.f) != dg[u]) return fail(ETALE_EINVAL, "truncated lists");
        for (u32 j = 0; j < dg[u]; j++)
            if (slabh[at + j].x >= n) return fail(ETALE_EINVAL, "a list names an id beyond next_id");
        refh[u] = ref_pack(del, dg[u], (u32)k) | ((u64)((fl[u] >> 2) & 1u) << 56);
        k++;
        if (slabh.size() >= SNAP_CHUNK * R || u + 1 == n) {
            if (cudaMemcpy(idx->slab + kflush * R, slabh.data(), slabh.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(ETALE_ECUDA, "load slabs");
            kflush = k;
            slabh.clear();
        }
    }
    if (!slabh.empty() &&
        cudaMemcpy(idx->slab + kflush * R, slabh.data(), slabh.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ETALE_ECUDA, "load slabs");
    std::vector<u32> eh(ne);
    if (ne && fread(eh.data(), 4, ne, f.f) != ne) return fail(ETALE_EINVAL, "truncated entry set");
    for (u32 e : eh)
        if (e >= n) return fail(ETALE_EINVAL, "an entry id beyond next_id");
    const u64 free_n = idx->pool - used;
    if ((n && cudaMemcpy(idx->ref, refh.data(), n * 8, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(idx->ctr + C_FREE, &free_n, 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        (ne && cudaMemcpy(idx->entries, eh.data(), (size_t)ne * 4, cudaMemcpyHostToDevice) != cudaSuccess))
        return fail(ETALE_ECUDA, "load references");
    idx->next_id = n;
    idx->live = live;
    idx->tombs = tombs;
    idx->reclaimed = reclaimed;
    idx->free_lb = free_n;
    idx->n_entries = ne;
    cudaStream_t st = nullptr;
    if (launch_set_u32(idx->nent_dev, ne, st) != cudaSuccess ||
        launch_ingest_copies(idx->dev(), 0, n, st) != cudaSuccess)
        return fail(ETALE_ECUDA, "load copies");
    g_kernel_launches += 2;
    if (idx->seed_tc && ne) {
        const SeedTcPlan p = seed_tc_plan(idx->dim, ne, 0);
        if (!grow(idx->sd_E, p.bytes_E) || !grow(idx->sd_en, (size_t)p.s_pad * 4) || !grow(idx->sd_estat, 64))
            return fail(ETALE_ENOMEM, "entry-set copy");
        if (launch_seed_tc_entries(idx->dev(), ne, p, idx->seed_bufs(), st) != cudaSuccess)
            return fail(ETALE_ECUDA, "entry-set copy");
        g_kernel_launches++;
    }
    u64 inexact = 0;
    if (cudaMemcpy(&inexact, idx->ctr + C_INEXACT, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ETALE_ECUDA, "load synchronise");
    idx->rows_exact = inexact == 0;
    *out = idx;
    return ETALE_OK;
}

etale_status etale_set_writer_share(etale_index *idx, float share) {
    if (!idx) return ETALE_EINVAL;
    if (!(share > 0.f && share <= 1.f)) return idx->fail(ETALE_EINVAL, "share must be in (0, 1]");
    idx->writer_sms = std::max(1, (int)(idx->num_sms * share + 0.5f));
    return ETALE_OK;
}

etale_status etale_set_rerank(etale_index *idx, uint32_t rerank) {
    if (!idx) return ETALE_EINVAL;
    if (rerank == 0 || rerank > 256) return idx->fail(ETALE_EINVAL, "rerank must be 1..256");
    idx->cfg.rerank = rerank;
    return ETALE_OK;
}

etale_status etale_set_insert_precision(etale_index *idx, etale_precision p) {
    if (!idx) return ETALE_EINVAL;
    if (p == ETALE_PREC_BF16 && !idx->xb) return idx->fail(ETALE_EINVAL, "no bf16 copy kept (config.copies bit 0)");
    if (p == ETALE_PREC_FP8 && !idx->x8) return idx->fail(ETALE_EINVAL, "no fp8 copy kept (config.copies bit 1)");
    if ((u32)p > 2) return idx->fail(ETALE_EINVAL, "unknown precision");
    idx->insert_prec = (u32)p;
    return ETALE_OK;
}

etale_status etale_set_search_precision(etale_index *idx, etale_precision p) {
    if (!idx) return ETALE_EINVAL;
    if (p == ETALE_PREC_BF16 && !idx->xb) return idx->fail(ETALE_EINVAL, "no bf16 copy kept (config.copies bit 0)");
    if (p == ETALE_PREC_FP8 && !idx->x8) return idx->fail(ETALE_EINVAL, "no fp8 copy kept (config.copies bit 1)");
    if ((u32)p > 2) return idx->fail(ETALE_EINVAL, "unknown precision");
    idx->search_prec = (u32)p;
    return ETALE_OK;
}

etale_status etale_export_copies(etale_index *idx, uint64_t first, uint64_t n, uint16_t *bf16, uint8_t *fp8,
                                 float *scales) {
    if (!idx) return ETALE_EINVAL;
    if (first + n > idx->next_id) return idx->fail(ETALE_EINVAL, "range beyond next_id");
    if (n == 0) return ETALE_OK;
    if (bf16) {
        if (!idx->xb) return idx->fail(ETALE_EINVAL, "no bf16 copy kept");
        cudaError_t e = cudaMemcpy2D(bf16, (size_t)idx->dim * 2, idx->xb + first * idx->mb, (size_t)idx->mb * 2,
                                     (size_t)idx->dim * 2, n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return idx->cuda_fail(e, "export bf16");
    }
    if (fp8 || scales) {
        if (!idx->x8) return idx->fail(ETALE_EINVAL, "no fp8 copy kept");
        cudaError_t e = cudaSuccess;
        if (fp8)
            e = cudaMemcpy2D(fp8, idx->dim, idx->x8 + first * idx->m8, idx->m8, idx->dim, n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && scales) e = cudaMemcpy(scales, idx->x8s + first, n * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return idx->cuda_fail(e, "export fp8");
    }
    return ETALE_OK;
}

etale_status etale_set_profiling(etale_index *idx, int enable) {
    if (!idx) return ETALE_EINVAL;
    if (enable && idx->pev.empty()) {
        idx->pev.resize(2 * etale_index::MAXREC);
        for (auto &e : idx->pev)
            if (cudaEventCreate(&e) != cudaSuccess) return idx->cuda_fail(cudaGetLastError(), "event create");
    }
    idx->prof = enable != 0;
    idx->nrec = 0;
    return ETALE_OK;
}

static_assert((int)ETALE_WK_COUNT == (int)WK_N && (int)ETALE_WK_COMPACT == (int)WK_COMPACT,
              "work kinds of the header and the kernels differ");

etale_status etale_get_work(etale_index *idx, uint64_t *rows, uint64_t *state, uint32_t n, int reset) {
    if (!idx) return ETALE_EINVAL;
    if (n > ETALE_WK_COUNT) n = ETALE_WK_COUNT;
    u64 w[2 * WK_N];
    CK(cudaDeviceSynchronize(), "work tallies");
    CK(cudaMemcpy(w, idx->ctr + C_WK, sizeof(w), cudaMemcpyDeviceToHost), "work tallies");
    for (uint32_t i = 0; i < n; i++) {
        if (rows) rows[i] = w[2 * i];
        if (state) state[i] = w[2 * i + 1];
    }
    if (reset) CK(cudaMemset(idx->ctr + C_WK, 0, sizeof(w)), "work tallies");
    return ETALE_OK;
}

etale_status etale_get_profile(etale_index *idx, double *ms, uint64_t *count, uint32_t n, int reset) {
    if (!idx) return ETALE_EINVAL;
    if (n > ETALE_PH_COUNT) n = ETALE_PH_COUNT;
    for (uint32_t i = 0; i < n; i++) {
        if (ms) ms[i] = idx->pms[i];
        if (count) count[i] = idx->pcnt[i];
    }
    if (reset)
        for (int i = 0; i < ETALE_PH_COUNT; i++) { idx->pms[i] = 0; idx->pcnt[i] = 0; }
    return ETALE_OK;
}

}  // extern "C"
