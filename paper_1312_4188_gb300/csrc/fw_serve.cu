// Serving: continuous batching of classification requests against
// device-resident rule sets.
//
// The paper's prototype queues packets from the kernel to user space,
// accumulates a set, classifies it on the GPU and reinjects each packet with
// its verdict (Sec. IV, Fig. 1); it names asynchronous launches as the way to
// cut the delay further (Sec. V). Here requests (a packet batch for one rule
// set) arrive at any time. A scheduler thread owns a fixed number of slots
// (a stream, an event and a small device work list each) and, in copy mode, a
// device staging arena. Whenever a slot is free it admits the queued requests
// that fit -- at most max_group_requests requests and max_group_packets
// packets, and in copy mode arena space for their headers and verdicts -- and
// launches them together as one persistent batched kernel (fw_batch.cu). When
// a group's event completes, its slot and arena space are released at once,
// so requests that arrived meanwhile join the next launch while other groups
// are still running: several groups overlap on the device, and admission is
// bounded by free slots and free memory rather than by whole batches.
// Results are exactly fw_classify's for each request, alone or in a mix.
//
// Host cost per request is kept to a few tens of nanoseconds, below the
// device time of a typical request: requests live in a ring indexed by ticket
// (no allocation per request), the queue and every group are ranges of
// consecutive tickets, and each rule set's part of a work-list entry is
// built once, when the server starts.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fw_alloc.h"
#include "fw_batch.cuh"

namespace fwk {

static double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static size_t a16(size_t x) { return (x + 15) / 16 * 16; }

// Arena bytes of one copy-mode request: five header arrays and two verdict arrays.
static size_t request_bytes(int64_t n) {
    const size_t m = (size_t)n;
    return a16(4 * m) * 2 + a16(2 * m) * 2 + a16(m) + a16(4 * m) + a16(m);
}

// One request: an entry of the server's ring, at index ticket mod capacity (two cache lines).
struct alignas(64) SvRequest {
    uint64_t ticket = 0;    // 0: the entry is free (never used, or its ticket was released)
    int32_t set = 0;
    int32_t status = 1;     // 1 = not finished
    int64_t n = 0;
    // the request's buffers: in zero-copy mode their device-accessible aliases, in copy mode the
    // caller's host buffers
    fw_headers h{};
    int32_t *out_idx = nullptr;
    uint8_t *out_act = nullptr;
    double t_submit = 0, t_done = 0;
};
static_assert(sizeof(SvRequest) == 128, "a ring entry is two cache lines");

constexpr uint64_t kRingChunk = 1024;  // ring entries per allocation

struct SvSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    // the work list: the item counter (16 bytes), the jobs, then (16-byte aligned) the item
    // prefix; staged in pinned memory and copied in one piece, which also zeroes the counter
    unsigned char *d_work = nullptr;
    unsigned char *h_work = nullptr;
    bool busy = false;
    bool failed = false;  // the group's launch failed: it completes with FW_ECUDA
    uint64_t g_lo = 0, g_hi = 0;  // the group: tickets [g_lo, g_hi)
    int beside = 0;               // groups in flight when this one was admitted
    bool flip = false;            // the group takes the rule sets in reverse rank order
    int64_t packets = 0;          // the group's packets
    std::vector<uint32_t> order;  // the group's requests (offsets from g_lo) in job order
    std::vector<uint32_t> count;  // per set rank: requests of the group (then their first job)
    size_t arena_off = 0, arena_len = 0;
};

}  // namespace fwk

// A caller buffer registered for zero-copy use: [lo, hi) is device
// accessible at address + delta.
struct SvRange {
    uintptr_t lo, hi;
    intptr_t delta;
};

struct fw_server {
    fw_server_config cfg{};
    std::mutex reg_mu;
    std::vector<SvRange> ranges;
    std::vector<const fw_ruleset *> sets;
    int device = 0;
    int threads = 512;
    int32_t qcap = 256;
    uint8_t *d_arena = nullptr;
    size_t arena_bytes = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> length
    size_t arena_used = 0;
    std::vector<fwk::SvSlot> slots;
    std::vector<fwk::BatchJobDev> tmpl;  // per rule set: its work-list entry without buffers
    // rank of each rule set, costliest first (wider filter rows, then more reachable rules): a
    // group's jobs are ordered by it, so that items of one rule set run together and share the
    // L1-resident filter block
    std::vector<int32_t> set_rank;
    bool filter_only = false;            // every rule set has a bucket filter: k_batch_filter runs
    fwk::BatchFilterSet *d_fsets = nullptr;  // filter-only: the rule sets' filter blocks, by set index
    // Requests by ticket: entry t lives at ring index t & ring_mask, in chunks of kRingChunk
    // allocated when the server starts (addresses stay fixed). Tickets [admit_next, next_ticket) are
    // queued; an entry is reused only after its ticket was released by fw_server_wait.
    std::vector<fwk::SvRequest *> ring;
    uint64_t ring_mask = 0;
    uint64_t admit_next = 1;
    // a replay keeps the scheduler awake while it submits: the idle scheduler then polls the
    // submit counter (a cache line of its own, read without the lock) instead of sleeping
    alignas(64) std::atomic<uint64_t> enq_count{0};
    std::atomic<bool> hold_awake{false};
    std::atomic<bool> is_awake{false};
    char awake_pad[48];
    int64_t queued_packets = 0;  // packets of the queued requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    fw_server_stats stats{};
};

namespace fwk {

// The ring entry of ticket t; its chunk must exist.
static inline SvRequest &entry(fw_server *sv, uint64_t t) {
    const uint64_t i = t & sv->ring_mask;
    return sv->ring[i / kRingChunk][i % kRingChunk];
}

// The live request of a ticket, or nullptr (unknown or already released). Caller holds sv->mu.
static SvRequest *live_find(fw_server *sv, uint64_t ticket) {
    if (ticket == 0 || ticket >= sv->next_ticket) return nullptr;
    const uint64_t i = ticket & sv->ring_mask;
    SvRequest &e = sv->ring[i / kRingChunk][i % kRingChunk];
    return e.ticket == ticket ? &e : nullptr;
}

static bool arena_alloc(fw_server *sv, size_t len, size_t *off) {
    for (auto it = sv->free_blocks.begin(); it != sv->free_blocks.end(); ++it) {
        if (it->second < len) continue;
        *off = it->first;
        const size_t rest = it->second - len, roff = it->first + len;
        sv->free_blocks.erase(it);
        if (rest > 0) sv->free_blocks[roff] = rest;
        sv->arena_used += len;
        sv->stats.arena_high_water = std::max<int64_t>(sv->stats.arena_high_water, (int64_t)sv->arena_used);
        return true;
    }
    return false;
}

static void arena_free(fw_server *sv, size_t off, size_t len) {
    if (len == 0) return;
    sv->arena_used -= len;
    auto it = sv->free_blocks.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != sv->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        sv->free_blocks.erase(nx);
    }
    if (it != sv->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            sv->free_blocks.erase(it);
        }
    }
}

// Enqueue one group on its slot: (copy mode) header copies in, the work list,
// the persistent kernel, (copy mode) verdict copies out, the completion event.
static cudaError_t launch_group(fw_server *sv, SvSlot &sl) {
    const bool copy = sv->cfg.mode != FW_HOST_ZEROCOPY;
    int B = item_packets(sv->cfg.packets_per_item);
    if (sv->filter_only) {
        // filter items need no scan queue: a small group gets smaller items (down to 64 packets,
        // one step of a warp), about one for every warp of the launch, so its packets spread over
        // more warps and its latency falls; a large one keeps the configured size
        const int64_t warps = (int64_t)sm_count(sv->device) * kBatchFilterMinBlocks * (kBatchFilterThreads / 32);
        const int64_t want = (sl.packets + warps - 1) / warps;
        B = (int)std::min<int64_t>(B, std::max<int64_t>(64, (want + 63) / 64 * 64));
    }
    cudaError_t e = cudaSuccess;
    size_t off = sl.arena_off;
    int64_t n_items = 0;
    const size_t nj = (size_t)(sl.g_hi - sl.g_lo);
    // job order: by set rank (a counting sort, stable within a set), every other group in reverse
    // rank order, so that the end of one group and the start of the next, which overlap on the
    // device, work on the same rule set
    const size_t ns = sv->set_rank.size();
    auto rank = [&](size_t i) {
        const size_t r = (size_t)sv->set_rank[(size_t)entry(sv, sl.g_lo + i).set];
        return sl.flip ? ns - 1 - r : r;
    };
    sl.count.assign(ns + 1, 0);
    for (size_t i = 0; i < nj; ++i) ++sl.count[rank(i) + 1];
    for (size_t k = 1; k <= ns; ++k) sl.count[k] += sl.count[k - 1];
    sl.order.resize(nj);
    for (size_t i = 0; i < nj; ++i) sl.order[sl.count[rank(i)]++] = (uint32_t)i;
    unsigned long long *h_next = reinterpret_cast<unsigned long long *>(sl.h_work);
    *h_next = 0;
    // filter-only: compact jobs indexing the server's set table; else full jobs from the templates
    const bool fo = sv->filter_only;
    BatchJobDev *h_jobs = reinterpret_cast<BatchJobDev *>(sl.h_work + 16);
    BatchFilterJob *h_fjobs = reinterpret_cast<BatchFilterJob *>(sl.h_work + 16);
    // the item prefix follows the group's jobs in the same staging buffer
    const size_t po = 16 + a16(nj * (fo ? sizeof(BatchFilterJob) : sizeof(BatchJobDev)));
    int64_t *h_prefix = reinterpret_cast<int64_t *>(sl.h_work + po);
    for (size_t i = 0; i < nj && e == cudaSuccess; ++i) {
        const SvRequest &r = entry(sv, sl.g_lo + sl.order[i]);
        fw_headers dh = r.h;
        int32_t *di = r.out_idx;
        uint8_t *da = r.out_act;
        if (copy) {
            const size_t m = (size_t)r.n;
            uint8_t *base = sv->d_arena + off;
            size_t o = 0;
            uint32_t *s = reinterpret_cast<uint32_t *>(base + o); o += a16(4 * m);
            uint32_t *d = reinterpret_cast<uint32_t *>(base + o); o += a16(4 * m);
            uint16_t *sp = reinterpret_cast<uint16_t *>(base + o); o += a16(2 * m);
            uint16_t *dp = reinterpret_cast<uint16_t *>(base + o); o += a16(2 * m);
            uint8_t *pr = base + o; o += a16(m);
            di = reinterpret_cast<int32_t *>(base + o); o += a16(4 * m);
            da = base + o; o += a16(m);
            off += o;
            e = cudaMemcpyAsync(s, r.h.src, 4 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d, r.h.dst, 4 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sp, r.h.sport, 2 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dp, r.h.dport, 2 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(pr, r.h.proto, m, cudaMemcpyHostToDevice, sl.st);
            dh = fw_headers{s, d, sp, dp, pr};
        }
        if (fo) {
            BatchFilterJob &J = h_fjobs[i];
            J.h = HdrPtrs{dh.src, dh.dst, dh.sport, dh.dport, dh.proto};
            J.out_idx = di;
            J.out_act = da;
            J.n = r.n;
            J.set = r.set;
            J.item_packets = B;
            J.vec = job_vector_loads(dh);
            J.pad = 0;
        } else {
            // the rule set's part comes from its template; only the buffers are per request
            BatchJobDev &J = h_jobs[i];
            J = sv->tmpl[(size_t)r.set];
            J.vec = job_vector_loads(dh);
            J.h = HdrPtrs{dh.src, dh.dst, dh.sport, dh.dport, dh.proto};
            J.n = r.n;
            J.out_idx = di;
            J.out_act = da;
            J.item_packets = B;
        }
        h_prefix[i] = n_items;
        n_items += (r.n + B - 1) / B;
    }
    h_prefix[nj] = n_items;
    // counter, jobs and item prefix in one copy
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.d_work, sl.h_work, po + (nj + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, sl.st);
    unsigned long long *d_next = reinterpret_cast<unsigned long long *>(sl.d_work);
    const int64_t *d_prefix = reinterpret_cast<const int64_t *>(sl.d_work + po);
    if (e == cudaSuccess) {
        const int wpb = (fo ? kBatchFilterThreads : sv->threads) / 32;
        const int per_sm = fo ? kBatchFilterMinBlocks : 2;
        // alone on the device a group takes every SM it can use (one item a warp: the lowest
        // latency); beside other groups a small one gets fewer blocks (each warp several items),
        // leaving SMs to them
        const int64_t per_block = (int64_t)wpb * (sl.beside > 0 ? sv->cfg.items_per_warp : 1);
        const int64_t blocks = std::max<int64_t>(
            1, std::min<int64_t>((int64_t)sm_count(sv->device) * per_sm, (n_items + per_block - 1) / per_block));
        if (fo)
            e = launch_batch_filter(reinterpret_cast<const BatchFilterJob *>(sl.d_work + 16), sv->d_fsets, d_prefix,
                                    (int32_t)nj, n_items, d_next, blocks, sl.st, kBatchFilterMinBlocks);
        else
            e = launch_batch(reinterpret_cast<const BatchJobDev *>(sl.d_work + 16), d_prefix, (int32_t)nj, n_items,
                             d_next, sv->qcap, sv->threads, blocks, sl.st);
    }
    if (copy) {
        for (size_t i = 0; i < nj && e == cudaSuccess; ++i) {
            const SvRequest &r = entry(sv, sl.g_lo + sl.order[i]);
            const int32_t *oi = fo ? h_fjobs[i].out_idx : h_jobs[i].out_idx;
            const uint8_t *oa = fo ? h_fjobs[i].out_act : h_jobs[i].out_act;
            e = cudaMemcpyAsync(r.out_idx, oi, 4 * (size_t)r.n, cudaMemcpyDeviceToHost, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r.out_act, oa, (size_t)r.n, cudaMemcpyDeviceToHost, sl.st);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.st);
    return e;
}

// The scheduler. State (queue, slots' groups, arena, stats) changes only
// under the mutex; every CUDA call (event queries, copies, launches) is made
// with the mutex released, so submitters are never held up by the device.
static void worker_loop(fw_server *sv) {
    cudaSetDevice(sv->device);
    const bool copy = sv->cfg.mode != FW_HOST_ZEROCOPY;
    const int ns = (int)sv->slots.size();
    std::vector<int> busy_idx, done_idx, launch_idx;
    std::vector<cudaError_t> qres(ns);
    std::unique_lock<std::mutex> lk(sv->mu);
    int64_t launch_ns = 0;  // time of the last launches, added under the lock
    for (;;) {
        const int64_t tc0 = now_ns();
        sv->stats.launch_ns += launch_ns;
        launch_ns = 0;
        busy_idx.clear();
        for (int i = 0; i < ns; ++i)
            if (sv->slots[i].busy) busy_idx.push_back(i);
        // 1. completion checks, unlocked (a busy slot is touched only by this thread)
        lk.unlock();
        for (int i : busy_idx) qres[i] = cudaEventQuery(sv->slots[i].ev);
        lk.lock();
        int busy = 0;
        for (int i : busy_idx) {
            SvSlot &sl = sv->slots[i];
            const cudaError_t q = qres[i];
            if (q == cudaErrorNotReady) {
                ++busy;
                continue;
            }
            if (q != cudaSuccess) cudaGetLastError();
            const double t = now_us();
            const bool ok = q == cudaSuccess && !sl.failed;
            int64_t pk = 0;
            for (uint64_t k = sl.g_lo; k < sl.g_hi; ++k) {
                SvRequest &r = entry(sv, k);
                r.t_done = t;
                r.status = ok ? FW_OK : FW_ECUDA;
                pk += r.n;
            }
            const int64_t cnt = (int64_t)(sl.g_hi - sl.g_lo);
            if (ok) {
                sv->stats.completed += cnt;
                sv->stats.packets += pk;
            } else {
                sv->stats.failed += cnt;
            }
            arena_free(sv, sl.arena_off, sl.arena_len);
            sl.arena_len = 0;
            sl.g_lo = sl.g_hi = 0;
            sl.busy = false;
            sl.failed = false;
            sv->cv_done.notify_all();
        }
        const int64_t ta0 = now_ns();
        sv->stats.complete_ns += ta0 - tc0;
        // 2. admission, locked: every free slot takes the queued requests that fit
        launch_idx.clear();
        for (int i = 0; i < ns && sv->admit_next < sv->next_ticket; ++i) {
            SvSlot &sl = sv->slots[i];
            if (sl.busy) continue;
            // enough groups in flight: let the queue grow into a full group (fewer, larger launches)
            if (busy >= sv->cfg.busy_groups && sv->queued_packets < sv->cfg.max_group_packets) break;
            const uint64_t queued = sv->next_ticket - sv->admit_next;
            uint64_t take = 0;
            size_t bytes = 0;
            int64_t pk = 0;
            while (take < queued && (int64_t)take < sv->cfg.max_group_requests) {
                const SvRequest &r = entry(sv, sv->admit_next + take);
                if (take > 0 && pk + r.n > sv->cfg.max_group_packets) break;
                pk += r.n;
                bytes += copy ? request_bytes(r.n) : 0;
                ++take;
            }
            size_t off = 0;
            if (copy) {
                while (take > 0 && !arena_alloc(sv, bytes, &off)) {
                    --take;  // not enough free memory: admit fewer
                    const int64_t n = entry(sv, sv->admit_next + take).n;
                    bytes -= request_bytes(n);
                    pk -= n;
                }
                if (take == 0) break;  // wait for memory to free up
            }
            sv->queued_packets -= pk;
            sl.g_lo = sv->admit_next;
            sl.g_hi = sv->admit_next + take;
            sl.beside = busy;
            sl.flip = (sv->stats.groups & 1) != 0;
            sl.packets = pk;
            sv->admit_next += take;
            sl.arena_off = off;
            sl.arena_len = copy ? bytes : 0;
            sl.busy = true;
            ++busy;
            sv->stats.groups += 1;
            sv->stats.max_group_requests = std::max<int64_t>(sv->stats.max_group_requests, (int64_t)take);
            launch_idx.push_back(i);
        }
        int inflight = 0;
        for (const SvSlot &sl : sv->slots) inflight += sl.busy ? 1 : 0;
        sv->stats.max_inflight_groups = std::max<int64_t>(sv->stats.max_inflight_groups, inflight);
        sv->stats.pending = (int64_t)(sv->next_ticket - sv->admit_next);
        // 3. launches, unlocked
        if (!launch_idx.empty()) {
            lk.unlock();
            for (int i : launch_idx) {
                SvSlot &sl = sv->slots[i];
                if (launch_group(sv, sl) != cudaSuccess) {
                    cudaGetLastError();
                    sl.failed = true;
                    cudaEventRecord(sl.ev, sl.st);  // the group completes, with an error status
                }
            }
            launch_ns = now_ns() - ta0;
            lk.lock();
            continue;
        }
        sv->stats.launch_ns += now_ns() - ta0;
        const bool queued = sv->admit_next < sv->next_ticket;
        if (sv->stop && !queued && busy == 0) break;
        if (busy == 0 && !queued) {
            if (sv->hold_awake.load(std::memory_order_acquire)) {
                sv->is_awake.store(true, std::memory_order_release);
                const uint64_t seen = sv->enq_count.load(std::memory_order_acquire);
                lk.unlock();
                while (sv->hold_awake.load(std::memory_order_acquire) &&
                       sv->enq_count.load(std::memory_order_acquire) == seen)
                    std::this_thread::yield();
                lk.lock();
            } else {
                sv->cv_work.wait(lk);
            }
        } else {
            if (sv->hold_awake.load(std::memory_order_relaxed)) sv->is_awake.store(true, std::memory_order_relaxed);
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
}

// Device-accessible alias of a caller buffer (device memory or pinned host memory), or nullptr.
static const void *device_alias(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

}  // namespace fwk

using namespace fwk;

extern "C" int fw_server_register_buffer(fw_server *sv, const void *p, size_t bytes) {
    if (sv == nullptr || p == nullptr || bytes == 0) return set_status(FW_EINVAL);
    const void *d0 = device_alias(p);
    const void *d1 = device_alias(static_cast<const uint8_t *>(p) + bytes - 1);
    const intptr_t delta0 = reinterpret_cast<intptr_t>(d0) - reinterpret_cast<intptr_t>(p);
    const intptr_t delta1 = reinterpret_cast<intptr_t>(d1) - reinterpret_cast<intptr_t>(p) - (intptr_t)(bytes - 1);
    if (d0 == nullptr || d1 == nullptr || delta0 != delta1) return set_status(FW_EINVAL);
    std::lock_guard<std::mutex> lk(sv->reg_mu);
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    sv->ranges.push_back(SvRange{a, a + bytes, delta0});
    return FW_OK;
}

extern "C" int fw_server_unregister_buffer(fw_server *sv, const void *p) {
    if (sv == nullptr) return set_status(FW_EINVAL);
    std::lock_guard<std::mutex> lk(sv->reg_mu);
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    for (size_t i = 0; i < sv->ranges.size(); ++i)
        if (sv->ranges[i].lo == a) {
            sv->ranges.erase(sv->ranges.begin() + (int64_t)i);
            return FW_OK;
        }
    return set_status(FW_EINVAL);
}

extern "C" void fw_server_destroy(fw_server *sv) {
    if (sv == nullptr) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->hold_awake.store(false, std::memory_order_release);
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (SvSlot &sl : sv->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        cudaFree(sl.d_work);
        cudaFreeHost(sl.h_work);
    }
    cudaFree(sv->d_arena);
    cudaFree(sv->d_fsets);
    for (SvRequest *c : sv->ring) delete[] c;
    delete sv;
}

extern "C" int fw_server_create(const fw_ruleset *const *sets, int n_sets, const fw_server_config *cfg_in,
                                fw_server **out) {
    if (out == nullptr) return set_status(FW_EINVAL);
    *out = nullptr;
    if (n_sets <= 0 || sets == nullptr) return set_status(FW_EINVAL);
    for (int i = 0; i < n_sets; ++i)
        if (sets[i] == nullptr) return set_status(FW_EINVAL);
    fw_server_config c;
    std::memset(&c, 0, sizeof(c));
    if (cfg_in) c = *cfg_in;
    if (c.mode == 0) c.mode = FW_HOST_COPY;
    if (c.mode != FW_HOST_COPY && c.mode != FW_HOST_ZEROCOPY) return set_status(FW_EINVAL);
    if (c.slots == 0) c.slots = 4;
    if (c.max_group_requests == 0) c.max_group_requests = 256;
    if (c.max_pending == 0) c.max_pending = 1 << 16;
    if (c.max_group_packets == 0) c.max_group_packets = int64_t(1) << 20;
    if (c.arena_bytes == 0) c.arena_bytes = int64_t(256) << 20;
    if (c.packets_per_item == 0) c.packets_per_item = 256;
    if (c.segment_rules == 0) c.segment_rules = 64;
    if (c.block_threads == 0) c.block_threads = 512;
    if (c.items_per_warp == 0) c.items_per_warp = 1;
    if (c.busy_groups == 0) c.busy_groups = 2;
    if (c.slots < 1 || c.slots > 16 || c.max_group_requests < 1 || c.max_pending < 1 || c.max_group_packets < 1 ||
        c.arena_bytes < 4096 || c.packets_per_item % 128 != 0 || c.packets_per_item > 4096 ||
        c.segment_rules % 4 != 0 || c.segment_rules < 4 || c.block_threads % 32 != 0 || c.block_threads > 1024 ||
        c.items_per_warp < 1 || c.busy_groups < 1)
        return set_status(FW_EINVAL);
    for (int32_t r : c.reserved)
        if (r != 0) return set_status(FW_EINVAL);
    const size_t smem = batch_smem_bytes(c.block_threads, c.packets_per_item);
    if (smem > 227 * 1024) return set_status(FW_EINVAL);
    fw_server *sv = new (std::nothrow) fw_server();
    if (sv == nullptr) return set_status(FW_ENOMEM);
    sv->cfg = c;
    sv->sets.assign(sets, sets + n_sets);
    cudaGetDevice(&sv->device);
    sv->threads = c.block_threads;
    sv->qcap = c.packets_per_item;
    // ring capacity: every queued request plus every request of the groups in flight
    uint64_t cap = kRingChunk;
    while (cap < (uint64_t)c.max_pending + (uint64_t)c.slots * (uint64_t)c.max_group_requests) cap *= 2;
    sv->ring.assign(cap / kRingChunk, nullptr);
    sv->ring_mask = cap - 1;
    bool ring_ok = true;
    for (SvRequest *&c : sv->ring) {  // allocated (and touched) now, not while requests arrive
        c = new (std::nothrow) SvRequest[kRingChunk];
        if (c == nullptr) ring_ok = false;
    }
    sv->tmpl.resize((size_t)n_sets);
    sv->filter_only = true;
    for (int i = 0; i < n_sets; ++i)
        if (sets[i]->filter_words == 0) sv->filter_only = false;
    {
        std::vector<int32_t> by_cost((size_t)n_sets);
        for (int i = 0; i < n_sets; ++i) by_cost[(size_t)i] = i;
        // a set without a filter scans its sub-lists: costlier than any filtered one
        auto width = [&](int i) { return sets[i]->filter_words > 0 ? sets[i]->filter_words : INT32_MAX; };
        std::stable_sort(by_cost.begin(), by_cost.end(), [&](int32_t a, int32_t b) {
            return width(a) != width(b) ? width(a) > width(b) : sets[a]->n_eff > sets[b]->n_eff;
        });
        sv->set_rank.resize((size_t)n_sets);
        for (int k = 0; k < n_sets; ++k) sv->set_rank[(size_t)by_cost[(size_t)k]] = k;
    }
    for (int i = 0; i < n_sets; ++i)
        fill_batch_job(sv->tmpl[(size_t)i], sets[i], fw_headers{}, 0, nullptr, nullptr, item_packets(c.packets_per_item),
                       c.segment_rules);
    cudaError_t e = ring_ok ? prepare_batch_kernel(smem) : cudaErrorMemoryAllocation;
    if (e == cudaSuccess && c.mode == FW_HOST_COPY) {
        sv->arena_bytes = (size_t)c.arena_bytes;
        e = dev_malloc(&sv->d_arena, sv->arena_bytes);
        sv->free_blocks[0] = sv->arena_bytes;
    }
    sv->slots.resize(c.slots);
    for (SvSlot &sl : sv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        const size_t work_bytes = 16 + a16(c.max_group_requests * std::max(sizeof(BatchJobDev), sizeof(BatchFilterJob))) +
                                  (c.max_group_requests + 1) * sizeof(int64_t);
        if (e == cudaSuccess) e = dev_malloc(&sl.d_work, work_bytes);
        if (e == cudaSuccess) e = pinned_malloc(&sl.h_work, work_bytes);
    }
    if (e == cudaSuccess && sv->filter_only) {
        std::vector<BatchFilterSet> fs((size_t)n_sets);
        for (int i = 0; i < n_sets; ++i) fs[(size_t)i] = batch_filter_set(sets[i]);
        e = dev_malloc(&sv->d_fsets, fs.size() * sizeof(BatchFilterSet));
        if (e == cudaSuccess) e = cudaMemcpy(sv->d_fsets, fs.data(), fs.size() * sizeof(BatchFilterSet), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        fw_server_destroy(sv);
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return FW_OK;
}

namespace fwk {

// A request checked and, in zero-copy mode, its buffers resolved to device-accessible aliases
// (one pass over the registered ranges), written to *r without touching the queue. hint[7]: per
// buffer, the registered range to try first (updated). The caller holds sv->reg_mu.
static int prepare_request(fw_server *sv, int set, const fw_headers *h, int64_t n, int32_t *out_idx,
                           uint8_t *out_act, SvRequest *r, size_t *hint) {
    if (h == nullptr || n < 1 || n > INT32_MAX) return FW_EINVAL;
    if (set < 0 || set >= (int)sv->sets.size()) return FW_EINVAL;
    if (!h->src || !h->dst || !h->sport || !h->dport || !h->proto || !out_idx || !out_act) return FW_EINVAL;
    if (n > sv->cfg.max_group_packets) return FW_ERANGE;
    r->set = set;
    r->h = *h;
    r->n = n;
    r->out_idx = out_idx;
    r->out_act = out_act;
    if (sv->cfg.mode == FW_HOST_ZEROCOPY) {
        const size_t m = (size_t)n;
        const void *p[7] = {h->src, h->dst, h->sport, h->dport, h->proto, out_idx, out_act};
        const size_t len[7] = {4 * m, 4 * m, 2 * m, 2 * m, m, 4 * m, m};
        const void *d[7] = {};
        int found = 0;
        const size_t nr = sv->ranges.size();
        for (int k = 0; k < 7; ++k) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(p[k]);
            // start at the range that held this buffer last time (a request's buffers usually lie
            // where the previous request's did)
            const size_t h0 = hint[k] < nr ? hint[k] : 0;
            for (size_t j = 0; j < nr; ++j) {
                const size_t i = h0 + j < nr ? h0 + j : h0 + j - nr;
                const SvRange &rg = sv->ranges[i];
                if (a >= rg.lo && a + len[k] <= rg.hi) {
                    d[k] = reinterpret_cast<const void *>(a + rg.delta);
                    hint[k] = i;
                    ++found;
                    break;
                }
            }
        }
        if (found < 7)
            for (int k = 0; k < 7; ++k)
                if (d[k] == nullptr) d[k] = device_alias(p[k]);  // not registered: looked up now
        for (int k = 0; k < 7; ++k)
            if (d[k] == nullptr) return FW_EINVAL;
        r->h = fw_headers{static_cast<const uint32_t *>(d[0]), static_cast<const uint32_t *>(d[1]),
                          static_cast<const uint16_t *>(d[2]), static_cast<const uint16_t *>(d[3]),
                          static_cast<const uint8_t *>(d[4])};
        r->out_idx = static_cast<int32_t *>(const_cast<void *>(d[5]));
        r->out_act = static_cast<uint8_t *>(const_cast<void *>(d[6]));
    } else if (request_bytes(n) > sv->arena_bytes) {
        return FW_ERANGE;
    }
    return FW_OK;
}

// Queue prepared requests, in order, under one lock. Returns how many were queued; when that is
// fewer than `count`, *why is FW_EBUSY (max_pending requests queued, or the next ticket's ring
// entry is still held by an unreleased ticket).
static int64_t enqueue_requests(fw_server *sv, const SvRequest *rs, int64_t count, uint64_t *tickets,
                                int64_t t_start_ns, int *why) {
    int64_t k = 0;
    *why = FW_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const double t = now_us();
        for (; k < count; ++k) {
            if ((int64_t)(sv->next_ticket - sv->admit_next) >= sv->cfg.max_pending) {
                *why = FW_EBUSY;
                break;
            }
            const uint64_t tk = sv->next_ticket;
            SvRequest &e = entry(sv, tk);
            if (e.ticket != 0) {
                *why = FW_EBUSY;
                break;
            }
            e = rs[k];
            e.ticket = tk;
            e.status = 1;
            e.t_submit = t;
            e.t_done = 0;
            sv->queued_packets += e.n;
            sv->next_ticket = tk + 1;
            sv->stats.submitted += 1;
            tickets[k] = tk;
        }
        sv->stats.submit_ns += now_ns() - t_start_ns;
        if (k > 0) sv->enq_count.fetch_add((uint64_t)k, std::memory_order_release);
    }
    if (k > 0) sv->cv_work.notify_one();
    return k;
}

}  // namespace fwk

extern "C" int fw_server_submit(fw_server *sv, int set, const fw_headers *h, int64_t n, int32_t *out_idx,
                                uint8_t *out_act, uint64_t *ticket) {
    if (sv == nullptr || ticket == nullptr) return set_status(FW_EINVAL);
    SvRequest r;
    size_t hint[7] = {};
    const int64_t t0 = now_ns();
    int s;
    {
        std::lock_guard<std::mutex> lk(sv->reg_mu);
        s = prepare_request(sv, set, h, n, out_idx, out_act, &r, hint);
    }
    if (s != FW_OK) return set_status(s);
    int why = FW_OK;
    if (enqueue_requests(sv, &r, 1, ticket, t0, &why) == 0) return set_status(why);
    return FW_OK;
}

extern "C" int fw_server_wait(fw_server *sv, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    if (sv == nullptr) return set_status(FW_EINVAL);
    std::unique_lock<std::mutex> lk(sv->mu);
    SvRequest *r = live_find(sv, ticket);
    if (r == nullptr) return set_status(FW_EINVAL);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (r->status == 1) {
        if (timeout_us < 0) {
            sv->cv_done.wait(lk);
        } else if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->status == 1) {
            return set_status(FW_ETIMEOUT);
        }
    }
    if (latency_us) *latency_us = r->t_done - r->t_submit;
    const int s = r->status;
    r->ticket = 0;  // released: the ring entry can take a new request
    return set_status(s);
}

extern "C" int fw_server_drain(fw_server *sv, int64_t timeout_us) {
    if (sv == nullptr) return set_status(FW_EINVAL);
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    auto idle = [&] {
        if (sv->admit_next < sv->next_ticket) return false;
        for (const SvSlot &sl : sv->slots)
            if (sl.busy) return false;
        return true;
    };
    while (!idle()) {
        if (timeout_us < 0) sv->cv_done.wait(lk);
        else if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !idle())
            return set_status(FW_ETIMEOUT);
    }
    return FW_OK;
}

extern "C" int fw_server_get_stats(fw_server *sv, fw_server_stats *st) {
    if (sv == nullptr || st == nullptr) return set_status(FW_EINVAL);
    std::lock_guard<std::mutex> lk(sv->mu);
    *st = sv->stats;
    st->pending = (int64_t)(sv->next_ticket - sv->admit_next);
    return FW_OK;
}

extern "C" int fw_server_replay(fw_server *sv, fw_request *reqs, int64_t n, int64_t timeout_us) {
    if (sv == nullptr || n < 0 || (n > 0 && reqs == nullptr)) return set_status(FW_EINVAL);
    std::vector<uint64_t> tickets((size_t)n, 0);
    // requests already due are prepared together (up to kBatch) and queued under one lock
    constexpr int64_t kBatch = 128;
    std::vector<SvRequest> batch((size_t)kBatch);
    std::vector<int64_t> batch_req((size_t)kBatch);
    std::vector<uint64_t> batch_tickets((size_t)kBatch);
    size_t hint[7] = {};
    // wake the scheduler and keep it polling while the requests are submitted, as under steady
    // traffic (waking a sleeping thread takes tens of microseconds); the clock starts once it is up
    sv->is_awake.store(false, std::memory_order_release);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->hold_awake.store(true, std::memory_order_release);
    }
    sv->cv_work.notify_one();
    for (const double w0 = now_us(); !sv->is_awake.load(std::memory_order_acquire) && now_us() - w0 < 20000.0;)
        std::this_thread::yield();
    const double t0 = now_us();
    // Open loop: every request is submitted at its arrival time; when the submitting thread is
    // behind, the requests already due go together.
    int64_t i = 0;
    while (i < n) {
        const double now = now_us();
        if (now < t0 + reqs[i].arrival_us) continue;
        int64_t j = i, nb = 0;
        int64_t t_mark = now_ns();
        std::unique_lock<std::mutex> rl(sv->reg_mu);  // one hold of the registrations for the batch
        while (j < n && (j == i || now >= t0 + reqs[j].arrival_us) && nb < kBatch) {
            fw_request &q = reqs[j];
            const int s = prepare_request(sv, q.set, &q.hdrs, q.n, q.out_rule_idx, q.out_action, &batch[(size_t)nb],
                                          hint);
            if (s != FW_OK) {
                q.status = s;  // refused: keeps its status and gets no ticket
            } else {
                batch_req[(size_t)nb++] = j;
            }
            ++j;
        }
        rl.unlock();
        int64_t done = 0;
        while (done < nb) {
            int why = FW_OK;
            const int64_t got =
                enqueue_requests(sv, batch.data() + done, nb - done, batch_tickets.data() + done, t_mark, &why);
            for (int64_t k = done; k < done + got; ++k) tickets[(size_t)batch_req[(size_t)k]] = batch_tickets[(size_t)k];
            done += got;
            t_mark = now_ns();
            if (got == 0) std::this_thread::yield();  // the queue is full: wait for room
        }
        i = j;
    }
    sv->hold_awake.store(false, std::memory_order_release);
    int worst = FW_OK;
    for (int64_t i2 = 0; i2 < n; ++i2) {
        fw_request &q = reqs[i2];
        if (tickets[(size_t)i2] == 0) {
            worst = q.status;
            continue;
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        const SvRequest *r = live_find(sv, tickets[(size_t)i2]);
        const double t_submit = r->t_submit;
        lk.unlock();
        double lat = 0;
        const int s = fw_server_wait(sv, tickets[(size_t)i2], timeout_us, &lat);
        q.status = s;
        // open-loop latency: from the scheduled arrival, not from the submit call
        q.latency_us = (t_submit + lat) - (t0 + q.arrival_us);
        q.submit_lag_us = t_submit - (t0 + q.arrival_us);
        if (s != FW_OK) worst = s;
    }
    return worst == FW_OK ? FW_OK : set_status(worst);
}
