// Host-ingress path: headers in host memory in, verdicts in host memory out.
//
// The paper's prototype accumulates a set of packets, copies them to device
// memory, launches, and copies the verdict array back before reinjecting
// (Sec. IV.A, Sec. IV.C, Fig. 1). Here a batch is cut into chunks that flow
// through several streams so that the copy of one chunk overlaps the scan of
// another (FW_HOST_COPY), or the scan kernels read the pinned host pages
// directly over the host link and write the verdicts straight back
// (FW_HOST_ZEROCOPY), which needs no staging at all.
#include <algorithm>
#include <cstring>

#include "fw_alloc.h"
#include "fw_internal.cuh"

struct fw_host_pipeline {
    int device = 0;
    int nstreams = 0;
    int64_t chunk = 0;
    cudaStream_t st[8] = {};
    uint32_t *d_src[8] = {};
    uint32_t *d_dst[8] = {};
    uint16_t *d_sport[8] = {};
    uint16_t *d_dport[8] = {};
    uint8_t *d_proto[8] = {};
    int32_t *d_idx[8] = {};
    uint8_t *d_act[8] = {};
};

using namespace fwk;

extern "C" void fw_host_pipeline_destroy(fw_host_pipeline *pl) {
    if (pl == nullptr) return;
    for (int s = 0; s < pl->nstreams; ++s) {
        if (pl->st[s]) cudaStreamSynchronize(pl->st[s]);
        cudaFree(pl->d_src[s]);
        cudaFree(pl->d_dst[s]);
        cudaFree(pl->d_sport[s]);
        cudaFree(pl->d_dport[s]);
        cudaFree(pl->d_proto[s]);
        cudaFree(pl->d_idx[s]);
        cudaFree(pl->d_act[s]);
        if (pl->st[s]) cudaStreamDestroy(pl->st[s]);
    }
    delete pl;
}

extern "C" int fw_host_pipeline_create(int64_t chunk_packets, int n_streams, fw_host_pipeline **out) {
    if (out == nullptr) return set_status(FW_EINVAL);
    *out = nullptr;
    if (chunk_packets < 0 || n_streams < 0 || n_streams > 8) return set_status(FW_EINVAL);
    fw_host_pipeline *pl = new (std::nothrow) fw_host_pipeline();
    if (pl == nullptr) return set_status(FW_ENOMEM);
    pl->chunk = chunk_packets > 0 ? (chunk_packets + 3) / 4 * 4 : (int64_t(1) << 22);
    pl->nstreams = n_streams > 0 ? n_streams : 3;
    cudaGetDevice(&pl->device);
    cudaError_t e = cudaSuccess;
    const size_t c = (size_t)pl->chunk;
    for (int s = 0; s < pl->nstreams && e == cudaSuccess; ++s) {
        e = cudaStreamCreateWithFlags(&pl->st[s], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = dev_malloc(&pl->d_src[s], c * 4);
        if (e == cudaSuccess) e = dev_malloc(&pl->d_dst[s], c * 4);
        if (e == cudaSuccess) e = dev_malloc(&pl->d_sport[s], c * 2);
        if (e == cudaSuccess) e = dev_malloc(&pl->d_dport[s], c * 2);
        if (e == cudaSuccess) e = dev_malloc(&pl->d_proto[s], c);
        if (e == cudaSuccess) e = dev_malloc(&pl->d_idx[s], c * 4);
        if (e == cudaSuccess) e = dev_malloc(&pl->d_act[s], c);
    }
    if (e != cudaSuccess) {
        fw_host_pipeline_destroy(pl);
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    *out = pl;
    return FW_OK;
}

// Device alias of a pinned host pointer, or nullptr if the memory is not pinned.
static const void *mapped(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
    return a.devicePointer;
}

extern "C" int fw_classify_host(fw_host_pipeline *pl, const fw_ruleset *rs, const fw_headers *hh, int64_t n,
                                int32_t *out_idx, uint8_t *out_act, int strategy, const fw_config *cfg) {
    if (pl == nullptr || rs == nullptr || n < 0 || n > INT32_MAX) return set_status(FW_EINVAL);
    if (n == 0) return FW_OK;
    if (hh == nullptr || !hh->src || !hh->dst || !hh->sport || !hh->dport || !hh->proto || !out_idx || !out_act)
        return set_status(FW_EINVAL);
    if (strategy == FW_HOST_ZEROCOPY) {
        fw_headers dh;
        dh.src = static_cast<const uint32_t *>(mapped(hh->src));
        dh.dst = static_cast<const uint32_t *>(mapped(hh->dst));
        dh.sport = static_cast<const uint16_t *>(mapped(hh->sport));
        dh.dport = static_cast<const uint16_t *>(mapped(hh->dport));
        dh.proto = static_cast<const uint8_t *>(mapped(hh->proto));
        int32_t *di = static_cast<int32_t *>(const_cast<void *>(mapped(out_idx)));
        uint8_t *da = static_cast<uint8_t *>(const_cast<void *>(mapped(out_act)));
        if (!dh.src || !dh.dst || !dh.sport || !dh.dport || !dh.proto || !di || !da) return set_status(FW_EINVAL);
        int s = fw_classify_ex(rs, &dh, n, di, da, pl->st[0], cfg);
        if (s != FW_OK) return s;
        return set_status(cuda_status(cudaStreamSynchronize(pl->st[0])));
    }
    if (strategy != FW_HOST_COPY) return set_status(FW_EINVAL);
    int64_t c = 0;
    for (int64_t off = 0; off < n; off += pl->chunk, ++c) {
        const int s = (int)(c % pl->nstreams);
        const int64_t m = std::min(pl->chunk, n - off);
        cudaStream_t st = pl->st[s];
        cudaError_t e = cudaMemcpyAsync(pl->d_src[s], hh->src + off, m * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pl->d_dst[s], hh->dst + off, m * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pl->d_sport[s], hh->sport + off, m * 2, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pl->d_dport[s], hh->dport + off, m * 2, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pl->d_proto[s], hh->proto + off, m, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return set_status(cuda_status(e));
        fw_headers dh{pl->d_src[s], pl->d_dst[s], pl->d_sport[s], pl->d_dport[s], pl->d_proto[s]};
        int rc = fw_classify_ex(rs, &dh, m, pl->d_idx[s], pl->d_act[s], st, cfg);
        if (rc != FW_OK) return rc;
        e = cudaMemcpyAsync(out_idx + off, pl->d_idx[s], m * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_act + off, pl->d_act[s], m, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return set_status(cuda_status(e));
    }
    for (int s = 0; s < pl->nstreams; ++s) {
        cudaError_t e = cudaStreamSynchronize(pl->st[s]);
        if (e != cudaSuccess) return set_status(cuda_status(e));
    }
    return FW_OK;
}
