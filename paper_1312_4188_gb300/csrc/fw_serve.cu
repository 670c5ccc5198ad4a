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
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fw_alloc.h"
#include "fw_batch.cuh"

namespace fwk {

static double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static size_t a16(size_t x) { return (x + 15) / 16 * 16; }

// Arena bytes of one copy-mode request: five header arrays and two verdict arrays.
static size_t request_bytes(int64_t n) {
    const size_t m = (size_t)n;
    return a16(4 * m) * 2 + a16(2 * m) * 2 + a16(m) + a16(4 * m) + a16(m);
}

struct SvRequest {
    uint64_t ticket = 0;
    int set = 0;
    fw_headers h{};         // caller's buffers
    int64_t n = 0;
    int32_t *out_idx = nullptr;
    uint8_t *out_act = nullptr;
    fw_headers dh{};        // zero-copy: device-accessible aliases of the caller's buffers
    int32_t *d_idx = nullptr;
    uint8_t *d_act = nullptr;
    size_t bytes = 0;       // copy mode arena bytes
    double t_submit = 0, t_done = 0;
    int status = 1;         // 1 = not finished
};

struct SvSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    BatchJobDev *d_jobs = nullptr;  // the work list: jobs, then (16-byte aligned) the item prefix
    unsigned long long *d_next = nullptr;
    BatchJobDev *h_jobs = nullptr;  // pinned staging of the work list
    bool busy = false;
    bool failed = false;  // the group's launch failed: it completes with FW_ECUDA
    std::vector<SvRequest *> group;
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
    std::deque<fwk::SvRequest *> pending;
    std::unordered_map<uint64_t, fwk::SvRequest *> live;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    fw_server_stats stats{};
};

namespace fwk {

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
    const int B = item_packets(sv->cfg.packets_per_item);
    cudaError_t e = cudaSuccess;
    size_t off = sl.arena_off;
    int64_t n_items = 0;
    // the item prefix follows the group's jobs in the same staging buffer
    const size_t po = a16(sl.group.size() * sizeof(BatchJobDev));
    int64_t *h_prefix = reinterpret_cast<int64_t *>(reinterpret_cast<uint8_t *>(sl.h_jobs) + po);
    for (size_t i = 0; i < sl.group.size() && e == cudaSuccess; ++i) {
        SvRequest *r = sl.group[i];
        fw_headers dh = r->dh;
        int32_t *di = r->d_idx;
        uint8_t *da = r->d_act;
        if (copy) {
            const size_t m = (size_t)r->n;
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
            e = cudaMemcpyAsync(s, r->h.src, 4 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d, r->h.dst, 4 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(sp, r->h.sport, 2 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dp, r->h.dport, 2 * m, cudaMemcpyHostToDevice, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(pr, r->h.proto, m, cudaMemcpyHostToDevice, sl.st);
            dh = fw_headers{s, d, sp, dp, pr};
        }
        fill_batch_job(sl.h_jobs[i], sv->sets[r->set], dh, r->n, di, da, B, sv->cfg.segment_rules);
        h_prefix[i] = n_items;
        n_items += (r->n + B - 1) / B;
    }
    h_prefix[sl.group.size()] = n_items;
    const size_t nj = sl.group.size();
    // jobs and item prefix in one copy
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.d_jobs, sl.h_jobs, po + (nj + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, sl.st);
    const int64_t *d_prefix = reinterpret_cast<const int64_t *>(reinterpret_cast<const uint8_t *>(sl.d_jobs) + po);
    if (e == cudaSuccess) {
        const int wpb = sv->threads / 32;
        const int64_t blocks =
            std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count(sv->device) * 2, (n_items + wpb - 1) / wpb));
        e = launch_batch(sl.d_jobs, d_prefix, (int32_t)nj, n_items, sl.d_next, sv->qcap, sv->threads, blocks, sl.st);
    }
    if (copy) {
        for (size_t i = 0; i < nj && e == cudaSuccess; ++i) {
            SvRequest *r = sl.group[i];
            const BatchJobDev &J = sl.h_jobs[i];
            e = cudaMemcpyAsync(r->out_idx, J.out_idx, 4 * (size_t)r->n, cudaMemcpyDeviceToHost, sl.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r->out_act, J.out_act, (size_t)r->n, cudaMemcpyDeviceToHost, sl.st);
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
    for (;;) {
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
            for (SvRequest *r : sl.group) {
                r->t_done = t;
                r->status = ok ? FW_OK : FW_ECUDA;
                if (ok) {
                    sv->stats.completed += 1;
                    sv->stats.packets += r->n;
                } else {
                    sv->stats.failed += 1;
                }
            }
            arena_free(sv, sl.arena_off, sl.arena_len);
            sl.arena_len = 0;
            sl.group.clear();
            sl.busy = false;
            sl.failed = false;
            sv->cv_done.notify_all();
        }
        // 2. admission, locked: every free slot takes the queued requests that fit
        launch_idx.clear();
        for (int i = 0; i < ns && !sv->pending.empty(); ++i) {
            SvSlot &sl = sv->slots[i];
            if (sl.busy) continue;
            size_t take = 0, bytes = 0;
            int64_t pk = 0;
            while (take < sv->pending.size() && (int64_t)take < sv->cfg.max_group_requests) {
                const SvRequest *r = sv->pending[take];
                if (take > 0 && pk + r->n > sv->cfg.max_group_packets) break;
                pk += r->n;
                bytes += r->bytes;
                ++take;
            }
            size_t off = 0;
            if (copy) {
                while (take > 0 && !arena_alloc(sv, bytes, &off)) {
                    --take;  // not enough free memory: admit fewer
                    bytes -= sv->pending[take]->bytes;
                }
                if (take == 0) break;  // wait for memory to free up
            }
            for (size_t k = 0; k < take; ++k) {
                sl.group.push_back(sv->pending.front());
                sv->pending.pop_front();
            }
            sl.arena_off = off;
            sl.arena_len = copy ? bytes : 0;
            sl.busy = true;
            ++busy;
            sv->stats.groups += 1;
            sv->stats.max_group_requests = std::max<int64_t>(sv->stats.max_group_requests, (int64_t)sl.group.size());
            launch_idx.push_back(i);
        }
        int inflight = 0;
        for (const SvSlot &sl : sv->slots) inflight += sl.busy ? 1 : 0;
        sv->stats.max_inflight_groups = std::max<int64_t>(sv->stats.max_inflight_groups, inflight);
        sv->stats.pending = (int64_t)sv->pending.size();
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
            lk.lock();
            continue;
        }
        if (sv->stop && sv->pending.empty() && busy == 0) break;
        if (busy == 0 && sv->pending.empty()) {
            sv->cv_work.wait(lk);
        } else {
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
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (SvSlot &sl : sv->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        cudaFree(sl.d_jobs);
        cudaFree(sl.d_next);
        cudaFreeHost(sl.h_jobs);
    }
    cudaFree(sv->d_arena);
    for (auto &kv : sv->live) delete kv.second;
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
    if (c.slots < 1 || c.slots > 16 || c.max_group_requests < 1 || c.max_pending < 1 || c.max_group_packets < 1 ||
        c.arena_bytes < 4096 || c.packets_per_item % 128 != 0 || c.packets_per_item > 4096 ||
        c.segment_rules % 4 != 0 || c.segment_rules < 4 || c.block_threads % 32 != 0 || c.block_threads > 1024)
        return set_status(FW_EINVAL);
    const size_t smem = batch_smem_bytes(c.block_threads, c.packets_per_item);
    if (smem > 227 * 1024) return set_status(FW_EINVAL);
    fw_server *sv = new (std::nothrow) fw_server();
    if (sv == nullptr) return set_status(FW_ENOMEM);
    sv->cfg = c;
    sv->sets.assign(sets, sets + n_sets);
    cudaGetDevice(&sv->device);
    sv->threads = c.block_threads;
    sv->qcap = c.packets_per_item;
    cudaError_t e = prepare_batch_kernel(smem);
    if (e == cudaSuccess && c.mode == FW_HOST_COPY) {
        sv->arena_bytes = (size_t)c.arena_bytes;
        e = dev_malloc(&sv->d_arena, sv->arena_bytes);
        sv->free_blocks[0] = sv->arena_bytes;
    }
    sv->slots.resize(c.slots);
    for (SvSlot &sl : sv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        const size_t work_bytes = a16(c.max_group_requests * sizeof(BatchJobDev)) + (c.max_group_requests + 1) * sizeof(int64_t);
        if (e == cudaSuccess) e = dev_malloc(&sl.d_jobs, work_bytes);
        if (e == cudaSuccess) e = dev_malloc(&sl.d_next, sizeof(unsigned long long));
        if (e == cudaSuccess) e = pinned_malloc(&sl.h_jobs, work_bytes);
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
// (one pass over the registered ranges under one lock), without touching the queue.
static int prepare_request(fw_server *sv, int set, const fw_headers *h, int64_t n, int32_t *out_idx,
                           uint8_t *out_act, SvRequest **out) {
    if (h == nullptr || n < 1 || n > INT32_MAX) return FW_EINVAL;
    if (set < 0 || set >= (int)sv->sets.size()) return FW_EINVAL;
    if (!h->src || !h->dst || !h->sport || !h->dport || !h->proto || !out_idx || !out_act) return FW_EINVAL;
    if (n > sv->cfg.max_group_packets) return FW_ERANGE;
    SvRequest *r = new (std::nothrow) SvRequest();
    if (r == nullptr) return FW_ENOMEM;
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
        {
            std::lock_guard<std::mutex> lk(sv->reg_mu);
            for (int k = 0; k < 7; ++k) {
                const uintptr_t a = reinterpret_cast<uintptr_t>(p[k]);
                for (const SvRange &rg : sv->ranges)
                    if (a >= rg.lo && a + len[k] <= rg.hi) {
                        d[k] = reinterpret_cast<const void *>(a + rg.delta);
                        ++found;
                        break;
                    }
            }
        }
        if (found < 7)
            for (int k = 0; k < 7; ++k)
                if (d[k] == nullptr) d[k] = device_alias(p[k]);  // not registered: looked up now
        r->dh = fw_headers{static_cast<const uint32_t *>(d[0]), static_cast<const uint32_t *>(d[1]),
                           static_cast<const uint16_t *>(d[2]), static_cast<const uint16_t *>(d[3]),
                           static_cast<const uint8_t *>(d[4])};
        r->d_idx = static_cast<int32_t *>(const_cast<void *>(d[5]));
        r->d_act = static_cast<uint8_t *>(const_cast<void *>(d[6]));
        for (int k = 0; k < 7; ++k)
            if (d[k] == nullptr) {
                delete r;
                return FW_EINVAL;
            }
    } else {
        r->bytes = request_bytes(n);
        if (r->bytes > sv->arena_bytes) {
            delete r;
            return FW_ERANGE;
        }
    }
    *out = r;
    return FW_OK;
}

// Queue prepared requests, in order, under one lock; returns how many were queued (the rest do
// not fit under max_pending and stay with the caller).
static int64_t enqueue_requests(fw_server *sv, SvRequest *const *rs, int64_t count, uint64_t *tickets) {
    int64_t k = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const double t = now_us();
        for (; k < count && (int64_t)sv->pending.size() < sv->cfg.max_pending; ++k) {
            SvRequest *r = rs[k];
            r->ticket = sv->next_ticket++;
            r->t_submit = t;
            sv->pending.push_back(r);
            sv->live[r->ticket] = r;
            sv->stats.submitted += 1;
            tickets[k] = r->ticket;
        }
    }
    if (k > 0) sv->cv_work.notify_one();
    return k;
}

}  // namespace fwk

extern "C" int fw_server_submit(fw_server *sv, int set, const fw_headers *h, int64_t n, int32_t *out_idx,
                                uint8_t *out_act, uint64_t *ticket) {
    if (sv == nullptr || ticket == nullptr) return set_status(FW_EINVAL);
    SvRequest *r = nullptr;
    const int s = prepare_request(sv, set, h, n, out_idx, out_act, &r);
    if (s != FW_OK) return set_status(s);
    if (enqueue_requests(sv, &r, 1, ticket) == 0) {
        delete r;
        return set_status(FW_EBUSY);
    }
    return FW_OK;
}

extern "C" int fw_server_wait(fw_server *sv, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    if (sv == nullptr) return set_status(FW_EINVAL);
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->live.find(ticket);
    if (it == sv->live.end()) return set_status(FW_EINVAL);
    SvRequest *r = it->second;
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
    sv->live.erase(it);
    delete r;
    return set_status(s);
}

extern "C" int fw_server_drain(fw_server *sv, int64_t timeout_us) {
    if (sv == nullptr) return set_status(FW_EINVAL);
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    auto idle = [&] {
        if (!sv->pending.empty()) return false;
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
    st->pending = (int64_t)sv->pending.size();
    return FW_OK;
}

extern "C" int fw_server_replay(fw_server *sv, fw_request *reqs, int64_t n, int64_t timeout_us) {
    if (sv == nullptr || n < 0 || (n > 0 && reqs == nullptr)) return set_status(FW_EINVAL);
    std::vector<uint64_t> tickets((size_t)n, 0);
    std::vector<SvRequest *> batch;
    const double t0 = now_us();
    // Open loop: every request is submitted at its arrival time; when the submitting thread is
    // behind, all requests already due are prepared and queued together (one queue lock).
    int64_t i = 0;
    while (i < n) {
        const double now = now_us();
        if (now < t0 + reqs[i].arrival_us) continue;
        int64_t j = i;
        batch.clear();
        while (j < n && (j == i || now >= t0 + reqs[j].arrival_us) && j - i < 1024) {
            fw_request &q = reqs[j];
            SvRequest *r = nullptr;
            const int s = prepare_request(sv, q.set, &q.hdrs, q.n, q.out_rule_idx, q.out_action, &r);
            if (s != FW_OK) {
                q.status = s;
                tickets[j] = 0;
                r = nullptr;
            }
            batch.push_back(r);
            ++j;
        }
        // queue the prepared ones in order (a refused request keeps its status and no ticket)
        int64_t k = 0;
        while (k < (int64_t)batch.size()) {
            if (batch[k] == nullptr) {
                ++k;
                continue;
            }
            int64_t e = k;
            while (e < (int64_t)batch.size() && batch[e] != nullptr) ++e;
            int64_t done = 0;
            while (done < e - k) {
                const int64_t got = enqueue_requests(sv, batch.data() + k + done, e - k - done, &tickets[i + k + done]);
                done += got;
                if (got == 0) std::this_thread::yield();  // the queue is full: wait for room
            }
            k = e;
        }
        i = j;
    }
    int worst = FW_OK;
    for (int64_t i2 = 0; i2 < n; ++i2) {
        fw_request &q = reqs[i2];
        if (tickets[i2] == 0) {
            worst = q.status;
            continue;
        }
        std::unique_lock<std::mutex> lk(sv->mu);
        SvRequest *r = sv->live[tickets[i2]];
        lk.unlock();
        const double t_submit = r->t_submit;
        double lat = 0;
        const int s = fw_server_wait(sv, tickets[i2], timeout_us, &lat);
        q.status = s;
        // open-loop latency: from the scheduled arrival, not from the submit call
        q.latency_us = (t_submit + lat) - (t0 + q.arrival_us);
        if (s != FW_OK) worst = s;
    }
    return worst == FW_OK ? FW_OK : set_status(worst);
}
