// Device request queue: continuous batching with the scheduling done on the
// device by one persistent kernel (see include/fw.h, "device request queue").
//
// The paper's prototype gathers packets, classifies the set in one launch and
// returns the verdicts (Sec. IV, Fig. 1), and its conclusions name
// asynchronous launches as the way to cut the per-batch delay (Sec. V). Here a
// launch serves any number of requests:
//
//  host  -- a ring of request entries in pinned host memory (one entry per
//           ticket) and, after the ring, a tail word: the host writes new
//           entries, then stores the next ticket into the tail (release) -->
//  feeder (warps 0..3 of the first block of the launch to start) -- warp 0
//           polls the tail; once it is past the feeder's head, the four warps
//           copy up to 128 new entries into a device request table (one entry
//           a thread), split each request into items (64 packets while the
//           ring holds few requests, 256 or 1,024 when more wait), and, after
//           one fence, write the items into a device item ring (one 64-bit
//           word each: the lap of its item ticket, the request's slot, the
//           chunk) -->
//  worker warps -- claim item tickets from a global counter, poll the item
//           word of their ticket's lap (relaxed loads, backing off), classify
//           its packets through the request's bucket filter (batch_filter_run,
//           the routine of the batched kernel, headers read from L2), and
//           count the request's items down with a release add; the warp that
//           finishes the last one stores the ticket into the request's
//           completion word in pinned host memory (release, system scope).
//
// Every wait is bounded by %globaltimer. The feeder gives up after idle_ns
// without a new request and, once the launch is life_ns old, stops taking
// requests; before it leaves for lack of work it announces "exiting" to the
// host, then looks at the tail once more and carries on if a request arrived
// meanwhile, so that a request submitted around that moment is in most cases
// either taken by this launch or seen by the host at its submit, which then
// launches the kernel again. (The host does not fence between its tail store
// and its look, which would cost a round trip over the host link per request;
// the rare request that both miss waits for the backstop:) the host also
// relaunches whenever a request has been pending for 50 us and the last launch
// has finished. Workers leave when the feeder has quit and their claimed ticket
// was not released; item and request state lives in device memory across
// launches, and a small kernel before each launch resets the claim counter to
// the released item count.
#include <cuda.h>  // driver types only: the one driver call used is resolved at run time

#include <atomic>
#include <chrono>
#include <cstring>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fw_alloc.h"
#include "fw_batch.cuh"

namespace fwk {

// Host ring entry (pinned host memory, read by the feeder); seq = its ticket. The entries of
// tickets below the tail word (one more entry after the ring) are published.
struct alignas(128) DqHostReq {
    uint64_t seq;
    int32_t set;
    int32_t vec;
    int64_t n;
    uint64_t src, dst, sport, dport, proto, out_idx, out_act;  // device-accessible addresses
};
static_assert(sizeof(DqHostReq) == 128, "one ring entry is one 128-byte line");

// Device copy of a request (its ring slot), written by the feeder before it writes the request's
// items; `remaining` is counted down by the workers.
struct alignas(128) DqReqDev {
    uint64_t src, dst, sport, dport, proto, out_idx, out_act;
    int64_t n;
    uint64_t ticket;
    int32_t set;
    int32_t vec;
    int32_t remaining;  // items not yet finished
    int32_t chunk;      // packets per item of this request
};

// One work item is one 64-bit word in the item ring: the lap of its item ticket g (g / ring
// size, 28 bits), the request's table slot (16 bits) and the chunk index (20 bits). A worker that
// holds ticket g waits for the word at g mod ring size to carry g's lap; one store publishes it.
typedef unsigned long long DqItem;
constexpr int kItemSlotBits = 16, kItemChunkBits = 20, kItemLapBits = 28;

__host__ __device__ inline unsigned long long dq_item(uint64_t lap, uint32_t slot, uint32_t chunk) {
    return ((lap & ((1ull << kItemLapBits) - 1)) << (kItemSlotBits + kItemChunkBits)) |
           ((unsigned long long)slot << kItemChunkBits) | chunk;
}

// Control block in pinned host memory, shared by the host and the kernel.
struct alignas(64) DqCtl {
    uint64_t state;  // kernel -> host: epoch << 2 | phase (1 running, 2 exiting, 3 gone)
    uint64_t stop;   // host -> kernel: finish and leave
    uint64_t idle_exits, life_exits, requests, items;  // the feeders' running totals
    uint64_t feed_ns, feeds;  // time the feeders spent taking requests, and how many times they took some
    uint64_t feed_read_ns;    // the part of feed_ns spent reading entries into the request table
    uint64_t pad[7];
};

// Device state that outlives a launch.
struct DqDev {
    unsigned long long claim;    // next item ticket handed to a worker
    unsigned long long pub;      // items released so far
    unsigned long long head;     // next request ticket the feeder reads
    unsigned long long started;  // blocks of this launch that started (the first feeds)
    unsigned quit;               // the feeder of this launch has left
    unsigned status;             // kDqWorkerTimeout
    unsigned long long work_ns;  // time workers spent on items (summed over warps, all launches)
    unsigned long long items_done;
};

constexpr unsigned kDqWorkerTimeout = 1u;  // a worker's wait for its item ran out
constexpr unsigned kDqBadEntry = 2u;       // a ring entry was not its ticket's, or out of range
// Set in a completion word when the request was not classified (a bad entry).
constexpr uint64_t kDoneError = 1ull << 63;
constexpr uint64_t kPhaseRunning = 1, kPhaseExiting = 2, kPhaseGone = 3;

struct DqParams {
    const DqHostReq *ring;
    const uint64_t *tail;  // host-written: the ticket after the last published entry
    uint64_t *done;  // per ring entry: the ticket of its last finished request
    DqCtl *ctl;
    DqDev *dev;
    DqReqDev *req;
    DqItem *items;
    const BatchFilterSet *fsets;
    uint64_t ring_mask, items_mask;
    int32_t items_log2;
    uint64_t epoch;
    uint64_t idle_ns, life_ns, worker_limit_ns;
    int32_t chunk;
    uint32_t poll_ns;
    uint32_t one;
    int32_t n_sets;
    int64_t max_n;  // largest request
};

__device__ __forceinline__ uint64_t ld_relaxed_sys(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint64_t *p, uint64_t v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// (no "memory" clobber: the item stores need no order among themselves, and as volatile asm they
// stay after the fence that precedes them)
__device__ __forceinline__ void st_relaxed_gpu(unsigned long long *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v));
}
__device__ __forceinline__ void st_release_gpu_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_sc_sys() { asm volatile("fence.sc.sys;" ::: "memory"); }
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ int atom_add_release_gpu(int *p, int v) {
    int old;
    asm volatile("atom.add.release.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu(const unsigned long long *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_gpu_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The feeder: warps 0..kFeedWarps-1 of the first block, one ring entry a thread per pass.
constexpr int kFeedWarps = 4;
constexpr int kFeedBatch = 32 * kFeedWarps;

// Named barrier 1 over the feeder warps. The threads reach it from divergent code (per-lane work
// of uneven length), so it is the non-aligned form, preceded by a reconvergence of the warp: the
// aligned form (bar.sync) requires every thread of a warp to execute it together.
__device__ __forceinline__ void feeder_sync() {
    __syncwarp();
    asm volatile("barrier.sync 1, %0;" ::"n"(kFeedBatch) : "memory");
}

// Warp 0 watches the host's tail (relaxed loads: polling must not invalidate the SM's L1) and
// decides each pass; once the tail is past `head`, one acquire fence orders what follows after the
// host's entries, and the feeder warps take up to kFeedBatch of them together: each thread copies
// one entry into the request table and counts its items, warp 0 lays out the items of the pass,
// and all threads write them, after one fence each.
__device__ __noinline__ void dq_feeder(const DqParams &p, int warp, int lane) {
    __shared__ int32_t s_k, s_chunk;           // entries of this pass (-1: leave), its item size
    __shared__ int32_t s_c[kFeedBatch];        // items of each entry
    __shared__ int32_t s_first[kFeedBatch + 1];  // first item of each entry; [kFeedBatch] = total
    // the launch parameters in registers (the memory clobbers of the strong operations below would
    // otherwise reload them on every use)
    DqItem *const items = p.items;
    DqReqDev *const req = p.req;
    const DqHostReq *const ring = p.ring;
    const uint64_t *const tailp = p.tail;
    DqCtl *const ctl = p.ctl;
    const uint64_t ring_mask = p.ring_mask, items_mask = p.items_mask, idle_ns = p.idle_ns, life_ns = p.life_ns;
    const uint64_t epoch = p.epoch;
    const int items_log2 = p.items_log2;
    const int32_t chunk = p.chunk;
    DqDev *const dev = p.dev;
    const int64_t max_n = p.max_n;
    const int32_t n_sets = p.n_sets;
    const int tid = 32 * warp + lane;
    // Every decision below that depends on the clock is taken by all lanes of a warp alike: the
    // clock is read by lane 0 and broadcast (lanes reading it themselves could fall on both sides
    // of a limit and leave the warp's shuffles unmatched).
    auto warp_ns = [lane]() {
        uint64_t t = 0;
        if (lane == 0) t = global_ns();
        return (uint64_t)__shfl_sync(0xFFFFFFFFu, (unsigned long long)t, 0);
    };
    uint64_t head = dev->head, pub = dev->pub;
    uint64_t fed_req = 0, fed_items = 0, feed_ns = 0, feeds = 0, feed_read_ns = 0;
    const uint64_t t_start = warp_ns();
    uint64_t t_work = t_start, t_pass = t_start, backlog = 0;
    uint32_t nap = 32;
    int why = 0;  // 1 idle, 2 life, 3 stop
    if (tid == 0) st_release_sys(&ctl->state, epoch << 2 | kPhaseRunning);
    for (;;) {
        if (warp == 0) {
            int k = 0;
            for (uint32_t it = 0;; ++it) {
                if ((it & 7u) == 0) {
                    uint64_t stop = 0;
                    if (lane == 0) stop = ld_relaxed_sys(&ctl->stop);
                    if (__shfl_sync(0xFFFFFFFFu, stop, 0) != 0) {
                        why = 3;
                        k = -1;
                        break;
                    }
                }
                uint64_t tail = 0;
                if (lane == 0) tail = ld_relaxed_sys(tailp);
                tail = __shfl_sync(0xFFFFFFFFu, tail, 0);
                const uint64_t now = warp_ns();
                const bool life = now - t_start > life_ns;
                if (tail > head && !life) {
                    nap = 32;
                    k = (int)min(tail - head, (uint64_t)kFeedBatch);
                    backlog = tail - head;
                    t_pass = now;
                    break;
                }
                if (!life && now - t_work <= idle_ns) {
                    // back off from 32 to 512 ns while idle: every poll reads the host's tail line
                    __nanosleep(nap);
                    nap = min(2u * nap, 512u);
                    continue;
                }
                // leaving: announce it, then look once more (a request that arrived meanwhile
                // keeps an idle launch going; the host relaunches after a launch that reached its
                // time limit)
                int resume = 0;
                if (lane == 0) {
                    st_release_sys(&ctl->state, epoch << 2 | kPhaseExiting);
                    fence_sc_sys();
                    if (!life && ld_relaxed_sys(tailp) > head) {
                        st_release_sys(&ctl->state, epoch << 2 | kPhaseRunning);
                        resume = 1;
                    }
                }
                if (__shfl_sync(0xFFFFFFFFu, resume, 0) == 0) {
                    why = life ? 2 : 1;
                    k = -1;
                    break;
                }
                t_work = warp_ns();
            }
            if (lane == 0) {
                if (k > 0) fence_acq_rel_sys();  // the host wrote the entries before the tail
                s_k = k;
                // Item size by the requests waiting in the host ring: a few, chunk_packets, so
                // that a lone request is spread over many warps; more than one pass, 16x (fewer
                // items to write and to claim when the device is the bottleneck); else 4x.
                s_chunk = backlog <= 8 ? chunk : backlog <= (uint64_t)kFeedBatch ? 4 * chunk : 16 * chunk;
            }
        }
        feeder_sync();
        const int k = s_k;
        if (k < 0) break;
        const int32_t chunk_k = s_chunk;
        // thread tid copies entry tid of the pass (four uncached 16-byte loads from host memory;
        // the host rewrites the entry on every lap of the ring)
        int32_t c = 0;
        if (tid < k) {
            const uint64_t t = head + (uint64_t)tid;
            const uint4 *w = reinterpret_cast<const uint4 *>(ring + (t & ring_mask));
            const uint4 w0 = __ldcv(w), w1 = __ldcv(w + 1), w2 = __ldcv(w + 2), w3 = __ldcv(w + 3),
                        w4 = __ldcv(w + 4);
            auto u64 = [](uint32_t lo, uint32_t hi) { return (uint64_t)lo | ((uint64_t)hi << 32); };
            const int64_t n = (int64_t)u64(w1.x, w1.y);
            // An entry that is not this ticket's, or out of range, is never classified: the
            // request completes at once with the error bit in its completion word.
            const bool good = u64(w0.x, w0.y) == t && n >= 1 && n <= max_n && w0.z < (uint32_t)n_sets;
            c = good ? (int32_t)((n + chunk_k - 1) / chunk_k) : 0;
            if (!good) {
                atomicOr(&dev->status, kDqBadEntry);
                fence_acq_rel_sys();
                st_release_sys(p.done + (t & ring_mask), t | kDoneError);
            }
            DqReqDev r;
            r.src = u64(w1.z, w1.w);
            r.dst = u64(w2.x, w2.y);
            r.sport = u64(w2.z, w2.w);
            r.dport = u64(w3.x, w3.y);
            r.proto = u64(w3.z, w3.w);
            r.out_idx = u64(w4.x, w4.y);
            r.out_act = u64(w4.z, w4.w);
            r.n = n;
            r.ticket = t;
            r.set = (int32_t)w0.z;
            r.vec = (int32_t)w0.w;
            r.remaining = c;
            r.chunk = chunk_k;
            req[t & ring_mask] = r;
        }
        s_c[tid] = c;
        fence_acq_rel_gpu();  // this thread's request table entry before any item that names it
        feeder_sync();
        if (warp == 0) {
            const uint64_t t_read = warp_ns();
            if (lane == 0) feed_read_ns += t_read - t_pass;
            // exclusive prefix of the items, four entries a lane
            const int32_t c0 = s_c[4 * lane], c1 = s_c[4 * lane + 1], c2 = s_c[4 * lane + 2], c3 = s_c[4 * lane + 3];
            const int32_t sum = c0 + c1 + c2 + c3;
            int32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += v;
            }
            const int32_t base = incl - sum;
            s_first[4 * lane] = base;
            s_first[4 * lane + 1] = base + c0;
            s_first[4 * lane + 2] = base + c0 + c1;
            s_first[4 * lane + 3] = base + c0 + c1 + c2;
            if (lane == 31) s_first[kFeedBatch] = incl;
        }
        feeder_sync();
        // item i of the pass goes to thread i mod kFeedBatch (consecutive threads, consecutive ring
        // words); a thread's entry cursor only moves forward (entries past k have no items)
        const int32_t total = s_first[kFeedBatch];
        for (int32_t i = tid, e = 0; i < total; i += kFeedBatch) {
            while (e + 1 < kFeedBatch && s_first[e + 1] <= i) ++e;
            const uint64_t g = pub + (uint64_t)i;
            st_relaxed_gpu(items + (g & items_mask), dq_item(g >> items_log2, (uint32_t)((head + (uint64_t)e) & ring_mask),
                                                            (uint32_t)(i - s_first[e])));
        }
        feeder_sync();  // s_* are rewritten by the next pass
        pub += (uint64_t)total;
        head += (uint64_t)k;
        const uint64_t t_now = warp_ns();
        if (warp == 0) t_work = t_now;
        if (tid == 0) {
            dev->pub = pub;
            dev->head = head;
            fed_req += (uint64_t)k;
            fed_items += (uint64_t)total;
            feed_ns += t_now - t_pass;
            ++feeds;
        }
    }
    if (tid == 0) {
        dev->pub = pub;
        dev->head = head;
        DqCtl *c = ctl;
        st_relaxed_sys(&c->requests, ld_relaxed_sys(&c->requests) + fed_req);
        st_relaxed_sys(&c->items, ld_relaxed_sys(&c->items) + fed_items);
        if (why == 1) st_relaxed_sys(&c->idle_exits, ld_relaxed_sys(&c->idle_exits) + 1);
        if (why == 2) st_relaxed_sys(&c->life_exits, ld_relaxed_sys(&c->life_exits) + 1);
        st_relaxed_sys(&c->feed_ns, ld_relaxed_sys(&c->feed_ns) + feed_ns);
        st_relaxed_sys(&c->feeds, ld_relaxed_sys(&c->feeds) + feeds);
        st_relaxed_sys(&c->feed_read_ns, ld_relaxed_sys(&c->feed_read_ns) + feed_read_ns);
        fence_acq_rel_gpu();
        st_release_gpu_u32(&dev->quit, 1u);
        st_release_sys(&c->state, epoch << 2 | kPhaseGone);
    }
}

// A worker: claim an item ticket, wait for its release, classify, count the request down.
__device__ __forceinline__ void dq_worker(const DqParams &p, int lane) {
    // per-warp totals for the statistics, kept in shared memory (registers go to the item routine)
    __shared__ unsigned long long s_work_ns[16], s_items[16], s_t_item[16];
    const int wid = threadIdx.x >> 5;
    if (lane == 0) s_work_ns[wid] = s_items[wid] = 0;
    unsigned long long g = 0;
    if (lane == 0) g = atomicAdd(&p.dev->claim, 1ull);
    for (;;) {
        int ok = 0;
        uint32_t slot = 0, chunk = 0;
        unsigned long long g_next = 0;
        if (lane == 0) {
            const DqItem *item = p.items + (g & p.items_mask);
            const uint64_t lap = (g >> p.items_log2) & ((1ull << kItemLapBits) - 1);
            const int lap_shift = kItemSlotBits + kItemChunkBits;
            uint64_t word = 0;
            uint64_t t0 = 0;
            uint32_t nap = 32;
            // Relaxed polls, and no acquire once the item is there: an acquire drops the SM's L1,
            // where the other warps keep the filter blocks. What the item leads to is read from L2
            // only (the request table entry, the headers), and only after the item word has
            // arrived, since its address comes from that word; the feeder wrote the entry to L2
            // before the item (fence), and the host wrote the headers before it submitted.
            for (uint32_t spin = 0;; ++spin) {
                word = ld_relaxed_gpu(item);
                if ((word >> lap_shift) == lap) {
                    ok = 1;
                    break;
                }
                if (ld_relaxed_gpu_u32(&p.dev->quit) != 0u) {
                    fence_acq_rel_gpu();
                    word = ld_relaxed_gpu(item);  // written before the feeder left?
                    ok = (word >> lap_shift) == lap;
                    if (ok) fence_acq_rel_gpu();
                    break;
                }
                if ((spin & 15u) == 15u) {
                    const uint64_t now = global_ns();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > p.worker_limit_ns) {
                        atomicOr(&p.dev->status, kDqWorkerTimeout);
                        break;
                    }
                }
                // back off from 32 ns to poll_ns: a warp that just finished looks again soon, an
                // idle one keeps its polls (L2 traffic beside the working warps) rare
                __nanosleep(nap);
                nap = min(2 * nap, p.poll_ns);
            }
            if (ok) {
                slot = (uint32_t)(word >> kItemChunkBits) & (uint32_t)p.ring_mask;
                chunk = (uint32_t)word & ((1u << kItemChunkBits) - 1);
                g_next = atomicAdd(&p.dev->claim, 1ull);  // the next claim overlaps this item
            }
        }
        if (__shfl_sync(0xFFFFFFFFu, ok, 0) == 0) {
            if (lane == 0 && s_items[wid] != 0) {
                atomicAdd(&p.dev->work_ns, s_work_ns[wid]);
                atomicAdd(&p.dev->items_done, s_items[wid]);
            }
            return;
        }
        if (lane == 0) s_t_item[wid] = global_ns();
        slot = __shfl_sync(0xFFFFFFFFu, slot, 0);
        chunk = __shfl_sync(0xFFFFFFFFu, chunk, 0);
        const DqReqDev *r = p.req + slot;
        BatchFilterJob J;
        auto ld64 = [](const uint64_t *q) { return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long *>(q)); };
        J.h.src = reinterpret_cast<const uint32_t *>(ld64(&r->src));
        J.h.dst = reinterpret_cast<const uint32_t *>(ld64(&r->dst));
        J.h.sport = reinterpret_cast<const uint16_t *>(ld64(&r->sport));
        J.h.dport = reinterpret_cast<const uint16_t *>(ld64(&r->dport));
        J.h.proto = reinterpret_cast<const uint8_t *>(ld64(&r->proto));
        J.out_idx = reinterpret_cast<int32_t *>(ld64(&r->out_idx));
        J.out_act = reinterpret_cast<uint8_t *>(ld64(&r->out_act));
        J.n = (int64_t)ld64(reinterpret_cast<const uint64_t *>(&r->n));
        J.set = __ldcg(&r->set);
        J.vec = __ldcg(&r->vec);
        J.item_packets = __ldcg(&r->chunk);
        J.pad = 0;
        const uint64_t ticket = ld64(&r->ticket);
        BatchItem item;
        item.job = 0;
        item.start = (int64_t)chunk * J.item_packets;
        item.count = (int32_t)min((int64_t)J.item_packets, J.n - item.start);
        batch_filter_run<kBatchFilterPackets, true>(J, p.fsets[J.set], item, lane, p.one);
        __syncwarp();  // the lanes' verdicts before lane 0's release
        if (lane == 0) {
            if (atom_add_release_gpu(const_cast<int32_t *>(&r->remaining), -1) == 1) {
                fence_acq_rel_sys();  // every item's verdicts (seen through the count) before the ticket
                st_release_sys(p.done + slot, ticket);
            }
            s_work_ns[wid] += global_ns() - s_t_item[wid];
            s_items[wid] += 1;
        }
        g = g_next;
    }
}

// The first block of the launch to start feeds: its first kFeedWarps warps run the feeder, its
// other warps leave at once, so the feeder shares its SM with no more than the other resident
// blocks' warps. Every other warp works.
__global__ void __launch_bounds__(512, 2) k_dqueue(DqParams p) {
    __shared__ unsigned long long first;
    if (threadIdx.x == 0) first = atomicAdd(&p.dev->started, 1ull);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (first == 0) {
        if (threadIdx.x < kFeedBatch) dq_feeder(p, threadIdx.x >> 5, lane);
        return;
    }
    dq_worker(p, lane);
}

// Before each launch: claims restart at the released item count.
__global__ void k_dqueue_reset(DqDev *dev) {
    dev->claim = dev->pub;
    dev->started = 0;
    dev->quit = 0;
}

static double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct DqRange {
    uintptr_t lo, hi;
    intptr_t delta;
};

}  // namespace fwk

struct fw_dqueue {
    fw_dqueue_config cfg{};
    int device = 0;
    int grid = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_last = nullptr;  // recorded after the latest launch
    fwk::DqHostReq *ring = nullptr;  // pinned
    uint64_t *done = nullptr;        // pinned
    fwk::DqCtl *ctl = nullptr;       // pinned
    fwk::DqDev *d_dev = nullptr;
    fwk::DqReqDev *d_req = nullptr;
    fwk::DqItem *d_items = nullptr;
    fwk::BatchFilterSet *d_fsets = nullptr;
    uint64_t ring_n = 0, ring_mask = 0, items_n = 0, items_mask = 0;
    int32_t items_log2 = 0;
    std::vector<const fw_ruleset *> sets;
    std::mutex reg_mu;
    std::vector<fwk::DqRange> ranges;
    size_t hint[7] = {};  // fw_dqueue_submit's range hints (under reg_mu)
    std::mutex mu;  // the submitting side: next_ticket and the ring entries it writes
    uint64_t next_ticket = 1;
    // per ring entry: the ticket submitted and not yet released (0 = free); released by waiters
    // and the replay's poller without taking `mu`
    std::unique_ptr<std::atomic<uint64_t>[]> pending;
    std::vector<double> t_submit;    // per ring entry
    std::vector<int64_t> n_of;       // per ring entry: packets
    std::mutex launch_mu;
    // epochs launched; written under launch_mu, read without it by the submit and poll paths
    std::atomic<uint64_t> launched{0};
    std::atomic<bool> launch_failed{false};
    fwk::DqDev last_dev{};           // the device state as last read between launches
    // counters of the submitting side and of the completing side on cache lines of their own
    alignas(64) std::atomic<int64_t> submitted{0};
    std::atomic<int64_t> submit_ns{0};
    alignas(64) std::atomic<int64_t> completed{0};
    std::atomic<int64_t> packets{0};
    char counters_pad[48];
};

using namespace fwk;

namespace {

// Launch epoch `e` (reset kernel + persistent kernel) on the queue's stream. Caller holds launch_mu.
int dq_launch(fw_dqueue *q) {
    DqParams p;
    std::memset(&p, 0, sizeof(p));
    p.ring = q->ring;
    p.tail = &q->ring[q->ring_n].seq;
    p.done = q->done;
    p.ctl = q->ctl;
    p.dev = q->d_dev;
    p.req = q->d_req;
    p.items = q->d_items;
    p.fsets = q->d_fsets;
    p.ring_mask = q->ring_mask;
    p.items_mask = q->items_mask;
    p.items_log2 = q->items_log2;
    p.epoch = q->launched.load() + 1;
    p.idle_ns = (uint64_t)q->cfg.idle_us * 1000ull;
    p.life_ns = (uint64_t)q->cfg.life_ms * 1000000ull;
    p.worker_limit_ns = 4ull * p.life_ns + p.idle_ns;
    p.chunk = q->cfg.chunk_packets;
    p.n_sets = (int32_t)q->sets.size();
    p.max_n = q->cfg.max_request_packets;
    p.poll_ns = (uint32_t)q->cfg.poll_ns;
    p.one = 1;
    k_dqueue_reset<<<1, 1, 0, q->st>>>(q->d_dev);
    k_dqueue<<<(unsigned)q->grid, 512, 0, q->st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(q->ev_last, q->st);
    if (e != cudaSuccess) {
        q->launch_failed.store(true);
        return cuda_status(e);
    }
    q->launched.store(p.epoch);
    return FW_OK;
}

// Whether a launch is due: the latest launch announced that it leaves, or (check_event) it has
// finished while requests may be pending. -1 when the queue's launches failed.
int dq_need_launch(fw_dqueue *q, bool check_event) {
    if (q->launch_failed.load()) return -1;
    const uint64_t s = __atomic_load_n(&q->ctl->state, __ATOMIC_ACQUIRE);
    const uint64_t launched = q->launched.load();
    if (launched == 0 || ((s >> 2) == launched && (s & 3u) >= kPhaseExiting)) return 1;
    if (!check_event) return 0;
    const cudaError_t e = cudaEventQuery(q->ev_last);
    if (e == cudaSuccess) return 1;
    if (e != cudaErrorNotReady) {
        cudaGetLastError();
        q->launch_failed.store(true);
        return -1;
    }
    return 0;
}

// Launch the kernel again when it is due. The check runs without the lock (it is on every
// submit); a launch takes the lock and checks again.
int dq_kick(fw_dqueue *q, bool check_event) {
    int need = dq_need_launch(q, check_event);
    if (need == 0) return FW_OK;
    if (need < 0) return FW_ECUDA;
    std::lock_guard<std::mutex> lk(q->launch_mu);
    need = dq_need_launch(q, check_event);
    if (need <= 0) return need == 0 ? FW_OK : FW_ECUDA;
    int prev = q->device;
    cudaGetDevice(&prev);
    if (prev != q->device) cudaSetDevice(q->device);
    const int s2 = dq_launch(q);
    if (prev != q->device) cudaSetDevice(prev);
    return s2;
}

// Device-accessible alias of [p, p + bytes) when it lies in one registered range, else 0. The
// range that matched last for this argument (*hint) is tried first: a caller's requests usually
// come from the same few buffers.
uint64_t dq_alias(fw_dqueue *q, const void *p, size_t bytes, size_t *hint) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    if (a + bytes < a) return 0;
    const size_t nr = q->ranges.size();
    if (*hint < nr) {
        const DqRange &r = q->ranges[*hint];
        if (a >= r.lo && a + bytes <= r.hi) return (uint64_t)(a + r.delta);
    }
    for (size_t i = 0; i < nr; ++i) {
        const DqRange &r = q->ranges[i];
        if (a >= r.lo && a + bytes <= r.hi) {
            *hint = i;
            return (uint64_t)(a + r.delta);
        }
    }
    return 0;
}

// 0: not done; 1: done; -1: done without classification (the device found the entry bad).
int dq_done(const fw_dqueue *q, uint64_t slot, uint64_t ticket) {
    const uint64_t d = __atomic_load_n(&q->done[slot], __ATOMIC_ACQUIRE);
    if (d == ticket) return 1;
    return d == (ticket | kDoneError) ? -1 : 0;
}

void dq_release(fw_dqueue *q, uint64_t slot) { q->pending[slot].store(0, std::memory_order_release); }

void dq_free(fw_dqueue *q) {
    if (q->st) cudaStreamSynchronize(q->st);
    if (q->ev_last) cudaEventDestroy(q->ev_last);
    if (q->st) cudaStreamDestroy(q->st);
    if (q->ring) cudaFreeHost(q->ring);
    if (q->done) cudaFreeHost(q->done);
    if (q->ctl) cudaFreeHost(q->ctl);
    cudaFree(q->d_dev);
    cudaFree(q->d_req);
    cudaFree(q->d_items);
    cudaFree(q->d_fsets);
    cudaGetLastError();
    delete q;
}

}  // namespace

extern "C" int fw_dqueue_create(const fw_ruleset *const *sets, int n_sets, const fw_dqueue_config *cfg_in,
                                fw_dqueue **out) {
    if (out == nullptr) return set_status(FW_EINVAL);
    *out = nullptr;
    if (sets == nullptr || n_sets < 1 || n_sets > 65536) return set_status(FW_EINVAL);
    fw_dqueue_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in != nullptr) cfg = *cfg_in;
    for (int i = 0; i < 4; ++i)
        if (cfg.reserved[i] != 0) return set_status(FW_EINVAL);
    if (cfg.ring == 0) cfg.ring = 4096;
    if (cfg.chunk_packets == 0) cfg.chunk_packets = 64;
    if (cfg.blocks_per_sm == 0) cfg.blocks_per_sm = 2;
    if (cfg.idle_us == 0) cfg.idle_us = 1000;
    if (cfg.max_request_packets == 0) cfg.max_request_packets = 65536;
    if (cfg.life_ms == 0) cfg.life_ms = 2000;
    if (cfg.poll_ns == 0) cfg.poll_ns = 2048;
    if (cfg.ring < 64 || cfg.ring > 65536 || (cfg.ring & (cfg.ring - 1)) != 0) return set_status(FW_EINVAL);
    if (cfg.chunk_packets < 64 || cfg.chunk_packets % 64 != 0 || cfg.chunk_packets > (1 << 16))
        return set_status(FW_EINVAL);
    if (cfg.blocks_per_sm < 1 || cfg.blocks_per_sm > 2) return set_status(FW_EINVAL);
    if (cfg.idle_us < 1 || cfg.idle_us > 10000000 || cfg.life_ms < 1 || cfg.life_ms > 600000)
        return set_status(FW_EINVAL);
    if (cfg.poll_ns < 1 || cfg.poll_ns > 1000000 || cfg.max_request_packets < 1 ||
        cfg.max_request_packets > ((int64_t)1 << 31) - 1)
        return set_status(FW_EINVAL);
    for (int i = 0; i < n_sets; ++i)
        if (sets[i] == nullptr) return set_status(FW_EINVAL);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    for (int i = 0; i < n_sets; ++i)
        if (sets[i]->device != dev || sets[i]->filter_words == 0) return set_status(FW_EINVAL);
    const uint64_t per_req = (uint64_t)((cfg.max_request_packets + cfg.chunk_packets - 1) / cfg.chunk_packets);
    uint64_t items = 1;
    while (items < (uint64_t)cfg.ring * per_req) items <<= 1;
    if (items > (1ull << 26)) return set_status(FW_ERANGE);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    fw_dqueue *q = new fw_dqueue;
    q->cfg = cfg;
    q->device = dev;
    q->grid = sms * cfg.blocks_per_sm;
    q->ring_n = (uint64_t)cfg.ring;
    q->ring_mask = q->ring_n - 1;
    q->items_n = items;
    q->items_mask = items - 1;
    while ((1ull << q->items_log2) < items) ++q->items_log2;
    q->sets.assign(sets, sets + n_sets);
    q->pending.reset(new std::atomic<uint64_t>[q->ring_n]);
    for (uint64_t i = 0; i < q->ring_n; ++i) q->pending[i].store(0, std::memory_order_relaxed);
    q->t_submit.assign(q->ring_n, 0.0);
    q->n_of.assign(q->ring_n, 0);
    std::vector<BatchFilterSet> fs((size_t)n_sets);
    for (int i = 0; i < n_sets; ++i) fs[(size_t)i] = batch_filter_set(sets[i]);
    e = pinned_malloc(&q->ring, sizeof(DqHostReq) * (q->ring_n + 1));
    if (e == cudaSuccess) e = pinned_malloc(&q->done, sizeof(uint64_t) * q->ring_n);
    if (e == cudaSuccess) e = pinned_malloc(&q->ctl, sizeof(DqCtl));
    if (e == cudaSuccess) e = dev_malloc(&q->d_dev, sizeof(DqDev));
    if (e == cudaSuccess) e = dev_malloc(&q->d_req, sizeof(DqReqDev) * q->ring_n);
    if (e == cudaSuccess) e = dev_malloc(&q->d_items, sizeof(DqItem) * q->items_n);
    if (e == cudaSuccess) e = dev_malloc(&q->d_fsets, sizeof(BatchFilterSet) * (size_t)n_sets);
    if (e == cudaSuccess) {
        std::memset(q->ring, 0, sizeof(DqHostReq) * (q->ring_n + 1));
        std::memset(q->done, 0, sizeof(uint64_t) * q->ring_n);
        std::memset(q->ctl, 0, sizeof(DqCtl));
        DqDev d0;
        std::memset(&d0, 0, sizeof(d0));
        d0.head = 1;  // tickets start at 1
        e = cudaMemcpy(q->d_dev, &d0, sizeof(d0), cudaMemcpyHostToDevice);
    }
    // item words start with every lap bit set: lap 2^28 - 1 is reached after 2^28 laps of the ring
    if (e == cudaSuccess) e = cudaMemset(q->d_items, 0xFF, sizeof(DqItem) * q->items_n);
    if (e == cudaSuccess) e = cudaMemset(q->d_req, 0, sizeof(DqReqDev) * q->ring_n);
    if (e == cudaSuccess)
        e = cudaMemcpy(q->d_fsets, fs.data(), sizeof(BatchFilterSet) * (size_t)n_sets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ev_last, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        dq_free(q);
        return set_status(e == cudaErrorMemoryAllocation ? FW_ENOMEM : cuda_status(e));
    }
    *out = q;
    return set_status(FW_OK);
}

extern "C" void fw_dqueue_destroy(fw_dqueue *q) {
    if (q == nullptr) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(q->device);
    __atomic_store_n(&q->ctl->stop, 1ull, __ATOMIC_RELEASE);
    dq_free(q);
    cudaSetDevice(prev);
    cudaGetLastError();
}

namespace {

// The address range of the allocation holding device address a, as the driver records it
// (cuPointerGetAttribute: RANGE_START_ADDR, RANGE_SIZE), in [*lo, *hi). False when the driver
// gives no range for it.
bool alloc_range(uintptr_t a, uintptr_t *lo, uintptr_t *hi) {
    using GetAttr = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);
    static const GetAttr get = []() -> GetAttr {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult r = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &r) !=
                cudaSuccess ||
            r != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<GetAttr>(f);
    }();
    if (get == nullptr) return false;
    CUdeviceptr start = 0;
    size_t size = 0;
    if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)a) != CUDA_SUCCESS ||
        get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)a) != CUDA_SUCCESS || size == 0)
        return false;
    *lo = (uintptr_t)start;
    *hi = (uintptr_t)start + size;
    return true;
}

}  // namespace

extern "C" int fw_dqueue_register_buffer(fw_dqueue *q, const void *p, size_t bytes) {
    if (q == nullptr || p == nullptr || bytes == 0) return set_status(FW_EINVAL);
    const void *ends[2] = {p, static_cast<const uint8_t *>(p) + bytes - 1};
    intptr_t delta[2] = {0, 0};
    for (int k = 0; k < 2; ++k) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ends[k]) != cudaSuccess) {
            cudaGetLastError();
            return set_status(FW_EINVAL);
        }
        const void *d = nullptr;
        if ((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == q->device)
            d = ends[k];
        else if (a.type == cudaMemoryTypeHost)
            d = a.devicePointer;
        if (d == nullptr) return set_status(FW_EINVAL);
        delta[k] = reinterpret_cast<intptr_t>(d) - reinterpret_cast<intptr_t>(ends[k]);
    }
    if (delta[0] != delta[1]) return set_status(FW_EINVAL);
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    // both ends in one allocation: two allocations with the same mapping (device memory, or
    // pinned host memory under unified addressing) can have unmapped addresses between them
    uintptr_t lo = 0, hi = 0;
    const uintptr_t d0 = (uintptr_t)((intptr_t)a + delta[0]);
    if (alloc_range(d0, &lo, &hi) && (d0 < lo || bytes > hi - d0)) return set_status(FW_EINVAL);
    std::lock_guard<std::mutex> lk(q->reg_mu);
    q->ranges.push_back(DqRange{a, a + bytes, delta[0]});
    return set_status(FW_OK);
}

namespace {

// Check one request and fill its ring entry (all but seq) with device-accessible addresses.
// Caller holds reg_mu.
int dq_prepare(fw_dqueue *q, int set, const fw_headers *hdrs, int64_t n, int32_t *out_idx, uint8_t *out_act,
               DqHostReq *e, size_t (&hint)[7]) {
    if (set < 0 || set >= (int)q->sets.size() || hdrs == nullptr || n < 1 || out_idx == nullptr ||
        out_act == nullptr)
        return FW_EINVAL;
    if (n > q->cfg.max_request_packets) return FW_ERANGE;
    const size_t m = (size_t)n;
    const uint64_t a[7] = {dq_alias(q, hdrs->src, 4 * m, &hint[0]),   dq_alias(q, hdrs->dst, 4 * m, &hint[1]),
                           dq_alias(q, hdrs->sport, 2 * m, &hint[2]), dq_alias(q, hdrs->dport, 2 * m, &hint[3]),
                           dq_alias(q, hdrs->proto, m, &hint[4]),     dq_alias(q, out_idx, 4 * m, &hint[5]),
                           dq_alias(q, out_act, m, &hint[6])};
    for (int k = 0; k < 7; ++k)
        if (a[k] == 0) return FW_EINVAL;
    const fw_headers dh{reinterpret_cast<const uint32_t *>(a[0]), reinterpret_cast<const uint32_t *>(a[1]),
                        reinterpret_cast<const uint16_t *>(a[2]), reinterpret_cast<const uint16_t *>(a[3]),
                        reinterpret_cast<const uint8_t *>(a[4])};
    e->seq = 0;
    e->set = set;
    e->vec = job_vector_loads(dh);
    e->n = n;
    e->src = a[0];
    e->dst = a[1];
    e->sport = a[2];
    e->dport = a[3];
    e->proto = a[4];
    e->out_idx = a[5];
    e->out_act = a[6];
    return FW_OK;
}

// Publish prepared entries in ticket order; returns how many went out (fewer than k when the next
// ticket's ring entry is still held: FW_EBUSY for the rest). Their tickets go to tickets[].
int64_t dq_publish(fw_dqueue *q, const DqHostReq *es, int64_t k, uint64_t *tickets) {
    std::lock_guard<std::mutex> lk(q->mu);
    const double now = now_us();
    int64_t i = 0;
    for (; i < k; ++i) {
        const uint64_t t = q->next_ticket;
        const uint64_t slot = t & q->ring_mask;
        if (q->pending[slot].load(std::memory_order_acquire) != 0) break;
        DqHostReq *e = q->ring + slot;
        DqHostReq x = es[i];
        x.seq = t;
        std::memcpy(e, &x, sizeof(DqHostReq));
        q->pending[slot].store(t, std::memory_order_relaxed);
        q->t_submit[slot] = now;
        q->n_of[slot] = es[i].n;
        q->next_ticket = t + 1;
        tickets[i] = t;
    }
    if (i > 0) __atomic_store_n(&q->ring[q->ring_n].seq, q->next_ticket, __ATOMIC_RELEASE);  // after the entries
    return i;
}

}  // namespace

extern "C" int fw_dqueue_submit(fw_dqueue *q, int set, const fw_headers *hdrs, int64_t n, int32_t *out_rule_idx,
                                uint8_t *out_action, uint64_t *ticket) {
    if (q == nullptr || ticket == nullptr) return set_status(FW_EINVAL);
    const int64_t t0 = now_ns();
    DqHostReq e;
    int s;
    {
        std::lock_guard<std::mutex> lk(q->reg_mu);
        s = dq_prepare(q, set, hdrs, n, out_rule_idx, out_action, &e, q->hint);
    }
    if (s != FW_OK) return set_status(s);
    if (dq_publish(q, &e, 1, ticket) != 1) return set_status(FW_EBUSY);
    s = dq_kick(q, false);
    q->submitted.fetch_add(1, std::memory_order_relaxed);
    q->submit_ns.fetch_add(now_ns() - t0, std::memory_order_relaxed);
    return set_status(s);
}

extern "C" int fw_dqueue_wait(fw_dqueue *q, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    if (q == nullptr || ticket == 0) return set_status(FW_EINVAL);
    const uint64_t slot = ticket & q->ring_mask;
    if (q->pending[slot].load(std::memory_order_acquire) != ticket) return set_status(FW_EINVAL);
    const double t0 = now_us();
    double t_check = t0;
    int dn;
    while ((dn = dq_done(q, slot, ticket)) == 0) {
        const double now = now_us();
        if (now - t_check > 50.0) {  // backstop: relaunch if the kernel has left with work pending
            t_check = now;
            const int s = dq_kick(q, true);
            if (s != FW_OK) return set_status(s);
        }
        if (timeout_us >= 0 && now - t0 > (double)timeout_us) return set_status(FW_ETIMEOUT);
    }
    const double t_done = now_us();
    if (latency_us != nullptr) *latency_us = t_done - q->t_submit[slot];
    q->completed.fetch_add(1, std::memory_order_relaxed);
    q->packets.fetch_add(q->n_of[slot], std::memory_order_relaxed);
    dq_release(q, slot);
    return set_status(dn > 0 ? FW_OK : FW_ECUDA);
}

extern "C" int fw_dqueue_get_stats(fw_dqueue *q, fw_dqueue_stats *st) {
    if (q == nullptr || st == nullptr) return set_status(FW_EINVAL);
    std::memset(st, 0, sizeof(*st));
    st->submitted = q->submitted.load();
    st->completed = q->completed.load();
    st->packets = q->packets.load();
    {
        std::lock_guard<std::mutex> lk(q->launch_mu);
        st->launches = (int64_t)q->launched.load();
    }
    st->idle_exits = (int64_t)__atomic_load_n(&q->ctl->idle_exits, __ATOMIC_ACQUIRE);
    st->life_exits = (int64_t)__atomic_load_n(&q->ctl->life_exits, __ATOMIC_ACQUIRE);
    st->fed_requests = (int64_t)__atomic_load_n(&q->ctl->requests, __ATOMIC_ACQUIRE);
    st->fed_items = (int64_t)__atomic_load_n(&q->ctl->items, __ATOMIC_ACQUIRE);
    st->feed_ns = (int64_t)__atomic_load_n(&q->ctl->feed_ns, __ATOMIC_ACQUIRE);
    st->feeds = (int64_t)__atomic_load_n(&q->ctl->feeds, __ATOMIC_ACQUIRE);
    st->feed_read_ns = (int64_t)__atomic_load_n(&q->ctl->feed_read_ns, __ATOMIC_ACQUIRE);
    // the device state is read between launches only (the copy does not wait for the queue's
    // stream, which does not synchronise with other streams)
    {
        std::lock_guard<std::mutex> lk(q->launch_mu);
        DqDev d;
        if (cudaEventQuery(q->ev_last) == cudaSuccess &&
            cudaMemcpy(&d, q->d_dev, sizeof(d), cudaMemcpyDeviceToHost) == cudaSuccess)
            q->last_dev = d;
        st->device_status = q->last_dev.status;
        st->work_ns = (int64_t)q->last_dev.work_ns;
        st->items_done = (int64_t)q->last_dev.items_done;
    }
    cudaGetLastError();
    st->submit_ns = q->submit_ns.load();
    return set_status(FW_OK);
}

extern "C" int fw_dqueue_replay(fw_dqueue *q, fw_request *reqs, int64_t n, int64_t timeout_us) {
    if (q == nullptr || n < 0 || (n > 0 && reqs == nullptr)) return set_status(FW_EINVAL);
    std::vector<uint64_t> tickets((size_t)n, 0);
    std::vector<double> t_sub((size_t)n, 0.0), t_done((size_t)n, 0.0);
    std::atomic<int64_t> n_sub{0};  // requests handed to the poller (submitted or refused), in order
    std::atomic<bool> gave_up{false};
    const double t0 = now_us();
    // the poller records each completion when it happens and releases its ticket
    std::thread poller([&]() {
        int64_t lo = 0;
        double last_progress = now_us(), t_check = last_progress;
        while (lo < n) {
            const int64_t hi = n_sub.load(std::memory_order_acquire);
            bool progress = false;
            for (int64_t i = lo; i < hi; ++i) {
                if (t_done[(size_t)i] != 0.0 || tickets[(size_t)i] == 0) continue;
                const uint64_t slot = tickets[(size_t)i] & q->ring_mask;
                const int dn = dq_done(q, slot, tickets[(size_t)i]);
                if (dn != 0) {
                    if (dn < 0) reqs[i].status = FW_ECUDA;
                    t_done[(size_t)i] = now_us();
                    q->completed.fetch_add(1, std::memory_order_relaxed);
                    q->packets.fetch_add(reqs[i].n, std::memory_order_relaxed);
                    dq_release(q, slot);
                    progress = true;
                }
            }
            while (lo < hi && (tickets[(size_t)lo] == 0 || t_done[(size_t)lo] != 0.0)) ++lo;
            const double now = now_us();
            if (progress) last_progress = now;
            if (lo < hi && now - t_check > 50.0) {
                t_check = now;
                if (dq_kick(q, true) != FW_OK) {
                    gave_up.store(true);
                    return;
                }
            }
            if (timeout_us >= 0 && lo < hi && now - last_progress > (double)timeout_us) {
                gave_up.store(true);
                return;
            }
            if (lo >= hi && gave_up.load()) return;
        }
    });
    // Open loop: every request is submitted at its arrival time; when the submitting thread is
    // behind, the requests already due are prepared together and published in one pass.
    constexpr int64_t kBatch = 64;
    size_t hint[7] = {};
    DqHostReq batch[kBatch];
    int64_t batch_req[kBatch];
    uint64_t batch_tickets[kBatch];
    int64_t i = 0;
    while (i < n && !gave_up.load(std::memory_order_relaxed)) {
        const double now = now_us();
        if (now < t0 + reqs[i].arrival_us) continue;
        const int64_t c0 = now_ns();
        int64_t j = i, nb = 0;
        {
            std::lock_guard<std::mutex> lk(q->reg_mu);
            while (j < n && nb < kBatch && (j == i || now >= t0 + reqs[j].arrival_us)) {
                fw_request &r = reqs[j];
                r.status = dq_prepare(q, r.set, &r.hdrs, r.n, r.out_rule_idx, r.out_action, &batch[nb], hint);
                if (r.status == FW_OK) batch_req[nb++] = j;
                ++j;
            }
        }
        int64_t done = 0;
        while (done < nb && !gave_up.load(std::memory_order_relaxed)) {
            const int64_t got = dq_publish(q, batch + done, nb - done, batch_tickets + done);
            if (got > 0) {
                const double ts = now_us();
                for (int64_t k = done; k < done + got; ++k) {
                    tickets[(size_t)batch_req[k]] = batch_tickets[k];
                    t_sub[(size_t)batch_req[k]] = ts;
                }
                done += got;
                q->submitted.fetch_add(got, std::memory_order_relaxed);
                if (dq_kick(q, false) != FW_OK) gave_up.store(true);
            } else {
                std::this_thread::yield();  // the next ticket's ring entry is still held: wait for the poller
            }
        }
        for (int64_t k = done; k < nb; ++k) reqs[batch_req[k]].status = FW_ETIMEOUT;
        q->submit_ns.fetch_add(now_ns() - c0, std::memory_order_relaxed);
        i = j;
        n_sub.store(i, std::memory_order_release);
    }
    if (i < n) {
        gave_up.store(true);
        n_sub.store(i, std::memory_order_release);
    }
    poller.join();
    int worst = FW_OK;
    for (int64_t k = 0; k < n; ++k) {
        fw_request &r = reqs[k];
        if (k >= i) r.status = FW_ETIMEOUT;
        if (r.status == FW_OK && t_done[(size_t)k] == 0.0) r.status = FW_ETIMEOUT;
        if (r.status == FW_OK) {
            r.latency_us = t_done[(size_t)k] - (t0 + r.arrival_us);
            r.submit_lag_us = t_sub[(size_t)k] - (t0 + r.arrival_us);
        }
        if (r.status != FW_OK) worst = r.status;
    }
    return worst == FW_OK ? set_status(FW_OK) : set_status(worst);
}
