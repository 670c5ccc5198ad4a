// Learned-index decomposition classifier (interval decomposition per field,
// rule bitmaps, AND, first set bit).
//
// Every field of a rule is an interval of that field's key space (Sec. IV
// rule model: a prefix is an address interval, a port range an interval, a
// protocol one value or all of them). Cutting each field's key space at every
// interval endpoint gives "elementary intervals" inside which no rule's
// field test changes. Rules are split by the same partition as the scan's
// (protocol class and, where it shortens the lists, the top bits of one
// address): per class, the sub-list of rules that can match a packet of that
// class, in list order. For class c, field f (src, dst, sport,
// dport) and elementary interval j, the row bits_{c,f}[j] has bit b set
// exactly when the b-th rule of c's sub-list covers interval j in field f. A
// packet of class c lies in that rule iff bit b is set in the rows of its four
// fields' intervals, so the first match (Sec. I) is the rule behind the lowest
// set bit of the AND of four rows, found by scanning words from the start.
// The sub-list holds every rule that can match the packet, in order, so the
// answer is the whole list's first match. When more exact protocols are in use
// than there are protocol classes, the "other" classes hold rules of several
// protocols and get protocol rows too, ANDed as a fifth row.
//
// Locating a key's elementary interval: a piecewise-linear FP32 model per
// field (the key space cut into `segments` equal parts, one line per part fit
// on the sorted endpoints: least squares or the chord, whichever has the
// smaller exact error bound) predicts the position; the stored
// per-part maximum error bounds an exact integer binary search around it.
// The window is verified with integer compares before it is trusted (a
// failed check falls back to a search over the whole array and is counted),
// so floating point never decides a match.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fw_alloc.h"
#include "fw_internal.cuh"
#include "fw_lindex_fit.h"

namespace fwk {

constexpr int kFields = 5;      // src, dst, sport, dport, proto (intervals and models)
constexpr int kRowFields = 4;   // fields with bitmap rows; the protocol (and key) select the class
constexpr int kKeyBits[kFields] = {32, 32, 16, 16, 8};

struct LiFieldDev {
    const uint32_t *bound;  // M sorted interval starts, bound[0] = 0
    const float4 *model;    // per segment {slope, intercept, max |prediction - position| (int bits), 0}
    int32_t M;
    int32_t shift;          // segment = key >> shift
};

// One class: its rows (per field, M_f rows of W words, in quads of four words:
// the uint4 holding words [4q, 4q+4) of row j sits at q * qs + j * js). Short
// rows (at most 4 quads) are stored row by row (qs = 1, js = quads), so a
// packet's quads are adjacent; long rows quad-major (qs = M_f, js = 1), so
// the first quads of all the field's rows form one compact slab that stays in
// L2 while the rest of the rows stay in HBM. Also the original rule index
// behind each bit (-1 past the sub-list). A class that holds rules of several
// exact protocols ("other", when more protocols are in use than there are
// protocol classes) also has protocol rows (bits[4]); for every other class
// the protocol test is implied by the class.
struct LiClassDev {
    const uint4 *bits[kFields];
    const int32_t *orig;
    int64_t W;              // words per row (multiple of 4)
};

// Rows of at most this many quads (512 rules of a class sub-list) are stored row by row; longer
// rows quad-major. On 100K rules x 64M packets: the index truncated at the first catch-all (rows of
// at most 3 quads) 2.34 ms row by row against 2.68 ms quad-major; the full index (rows of ~300
// quads) 9.70 ms row by row against 6.08 ms quad-major.
constexpr int64_t kRowMajorQuads = 4;
__host__ __device__ inline bool li_row_major(int64_t W) { return W <= 4 * kRowMajorQuads; }

struct LiDev {
    LiFieldDev f[kFields];
    const LiClassDev *cls;  // n_classes entries (device memory)
    int32_t n_classes;
    int32_t key_field, key_bits;  // address key of the partition (part_class)
    const uint8_t *class_of;  // protocol -> protocol class (256 entries)
    const uint8_t *action;
    unsigned long long *fallbacks;
};

}  // namespace fwk

struct fw_lindex {
    int64_t n = 0, n_idx = 0, W = 0, first_catch_all = -1;
    int device = 0;
    int segments = 0;
    int64_t M[fwk::kFields] = {};
    int32_t max_err[fwk::kFields] = {};
    int64_t bitmap_bytes = 0;
    uint32_t *d_bound[fwk::kFields] = {};
    float4 *d_model[fwk::kFields] = {};
    int32_t shift[fwk::kFields] = {};
    int n_classes = 0, key_field = 0, key_bits = 0;
    uint32_t *d_bits[fwk::kMaxClasses][fwk::kFields] = {};
    int32_t *d_orig[fwk::kMaxClasses] = {};
    fwk::LiClassDev *d_cls = nullptr;
    uint8_t *d_class_of = nullptr;
    uint8_t *d_action = nullptr;
    unsigned long long *d_fallbacks = nullptr;
};

namespace fwk {

// ------------------------------------------------------------ device
// Quad q (words 4q..4q+3, rules 128q..128q+127 of the sub-list) of rows
// [j0, j0 + blockDim.x) of one field: the quad's 128 rule intervals are staged
// in shared memory and read by all lanes at once (broadcast); lane l computes
// the four words of row j0 + l and stores them as one uint4 at q * qs + (j0 + l) * js
// (contiguous across the warp when js = 1).
__global__ void k_li_build(const uint32_t *__restrict__ bound, int64_t M, const uint32_t *__restrict__ rlo,
                           const uint32_t *__restrict__ rhi, int64_t n_idx, int64_t Q, int64_t qs, int64_t js,
                           uint4 *__restrict__ bits) {
    __shared__ uint32_t slo[128], shi[128];
    const int64_t tiles = (M + blockDim.x - 1) / blockDim.x;
    for (int64_t t = blockIdx.x; t < Q * tiles; t += gridDim.x) {
        const int64_t q = t / tiles, j = (t % tiles) * blockDim.x + threadIdx.x;
        __syncthreads();
        for (int i = threadIdx.x; i < 128; i += blockDim.x) {
            const int64_t k = 128 * q + i;
            const bool ok = k < n_idx;
            slo[i] = ok ? rlo[k] : 1u;
            shi[i] = ok ? rhi[k] : 0u;  // empty interval: never covers
        }
        __syncthreads();
        if (j < M) {
            const uint32_t v = bound[j];
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                uint32_t word = 0;
#pragma unroll 8
                for (int b = 0; b < 32; ++b) word |= (uint32_t)((slo[32 * u + b] <= v) & (v <= shi[32 * u + b])) << b;
                w[u] = word;
            }
            bits[q * qs + j * js] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

template <bool SMEM>
__device__ __forceinline__ int li_locate(const LiFieldDev &f, const uint32_t *bound, uint32_t v,
                                         unsigned long long *fallbacks) {
    // shift is 32 for a one-segment address field: 64-bit shifts keep that defined (s = 0)
    const uint32_t s = (uint32_t)((uint64_t)v >> f.shift);
    const uint32_t base = (uint32_t)((uint64_t)s << f.shift);
    const float4 md = __ldg(f.model + s);
    const float pf = __fmaf_rn(md.x, __uint2float_rn(v - base), md.y);
    int p = (int)floorf(fminf(fmaxf(pf, 0.0f), (float)(f.M - 1)));
    const int e = __float_as_int(md.z);
    int lo = max(0, p - e), hi = min(f.M - 1, p + e);
    auto at = [&](int i) { return SMEM ? bound[i] : __ldg(bound + i); };
    // exact check of the window before it is trusted
    if (at(lo) > v || (hi < f.M - 1 && at(hi + 1) <= v)) {
        atomicAdd(fallbacks, 1ull);
        lo = 0;
        hi = f.M - 1;
    }
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (at(mid) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One packet per thread. The block first copies the class descriptors and,
// when they fit (SMEM), the four fields' interval starts into shared memory,
// which keeps the model windows and searches off the L1 path the rows use.
template <bool SMEM>
__global__ void __launch_bounds__(512) k_li_classify(LiDev d, const uint32_t *__restrict__ src,
                                                     const uint32_t *__restrict__ dst,
                                                     const uint16_t *__restrict__ sport,
                                                     const uint16_t *__restrict__ dport,
                                                     const uint8_t *__restrict__ proto, int64_t n,
                                                     int32_t *__restrict__ out_idx, uint8_t *__restrict__ out_act) {
    __shared__ LiClassDev scls[kMaxClasses];
    extern __shared__ __align__(16) uint32_t sbound[];
    if (threadIdx.x < d.n_classes) scls[threadIdx.x] = d.cls[threadIdx.x];
    const uint32_t *bound[kFields];
    int off = 0;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
        if (SMEM) {
            for (int i = threadIdx.x; i < d.f[f].M; i += blockDim.x) sbound[off + i] = __ldg(d.f[f].bound + i);
            bound[f] = sbound + off;
            off += d.f[f].M;
        } else {
            bound[f] = d.f[f].bound;
        }
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pr = proto[i];
        const uint32_t key[kRowFields] = {src[i], dst[i], sport[i], dport[i]};
        const LiClassDev &c = scls[part_class(__ldg(d.class_of + pr), d.key_field, d.key_bits, key[0], key[1])];
        const int64_t Q = c.W / 4;
        const bool rm = li_row_major(c.W);  // (quad q, row j) at q + j * Q, else at q * M_f + j
        const uint4 *row[kFields];
#pragma unroll
        for (int f = 0; f < kRowFields; ++f) {
            const int j = li_locate<SMEM>(d.f[f], bound[f], key[f], d.fallbacks);
            row[f] = c.bits[f] + (rm ? j * Q : (int64_t)j);
        }
        const bool prow = c.bits[kFields - 1] != nullptr;  // a class of mixed exact protocols
        row[kFields - 1] = nullptr;
        if (prow) {
            const int j = li_locate<SMEM>(d.f[kFields - 1], bound[kFields - 1], pr, d.fallbacks);
            row[kFields - 1] = c.bits[kFields - 1] + (rm ? j * Q : (int64_t)j);
        }
        int r = -1;
        for (int64_t q = 0; q < Q; ++q) {
            uint4 x = __ldg(row[0] + (rm ? q : q * d.f[0].M));
#pragma unroll
            for (int f = 1; f < kFields; ++f) {
                if (f == kFields - 1 && !prow) break;
                const uint4 y = __ldg(row[f] + (rm ? q : q * d.f[f].M));
                x.x &= y.x;
                x.y &= y.y;
                x.z &= y.z;
                x.w &= y.w;
            }
            if (x.x | x.y | x.z | x.w) {
                const int base = (int)(q * 128);
                const int bit = x.x ? base + __ffs(x.x) - 1
                              : x.y ? base + 32 + __ffs(x.y) - 1
                              : x.z ? base + 64 + __ffs(x.z) - 1
                                    : base + 96 + __ffs(x.w) - 1;
                r = __ldg(c.orig + bit);
                break;
            }
        }
        out_idx[i] = r;
        out_act[i] = r >= 0 ? __ldg(d.action + r) : (uint8_t)FW_DROP;
    }
}

// ------------------------------------------------------------ host
static void field_interval(const fw_rule &r, int f, uint32_t &lo, uint32_t &hi) {
    switch (f) {
        case 0: {
            const uint32_t m = prefix_mask(r.src_prefix);
            lo = r.src_addr & m;
            hi = lo | ~m;
            break;
        }
        case 1: {
            const uint32_t m = prefix_mask(r.dst_prefix);
            lo = r.dst_addr & m;
            hi = lo | ~m;
            break;
        }
        case 2: lo = r.sport_lo; hi = r.sport_hi; break;
        case 3: lo = r.dport_lo; hi = r.dport_hi; break;
        default:
            lo = r.proto_any ? 0u : r.proto;
            hi = r.proto_any ? 255u : r.proto;
    }
}

}  // namespace fwk

using namespace fwk;

extern "C" void fw_lindex_destroy(fw_lindex *li) {
    if (li == nullptr) return;
    for (int f = 0; f < kFields; ++f) {
        cudaFree(li->d_bound[f]);
        cudaFree(li->d_model[f]);
    }
    for (int c = 0; c < kMaxClasses; ++c) {
        for (int f = 0; f < kFields; ++f) cudaFree(li->d_bits[c][f]);
        cudaFree(li->d_orig[c]);
    }
    cudaFree(li->d_cls);
    cudaFree(li->d_class_of);
    cudaFree(li->d_action);
    cudaFree(li->d_fallbacks);
    delete li;
}

extern "C" int fw_lindex_create(const fw_rule *rules, int64_t n, const fw_lindex_config *cfg_in, fw_lindex **out) {
    if (out == nullptr) return set_status(FW_EINVAL);
    *out = nullptr;
    if (n < 0 || (n > 0 && rules == nullptr) || n > (int64_t(1) << 30)) return set_status(FW_EINVAL);
    fw_lindex_config cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    if (cfg_in) cfg = *cfg_in;
    const int segments = cfg.segments > 0 ? cfg.segments : 4096;
    if ((segments & (segments - 1)) != 0 || segments > (1 << 16)) return set_status(FW_EINVAL);
    if (cfg.truncate < 0 || cfg.truncate > 2) return set_status(FW_EINVAL);
    int64_t first_ca = -1;
    for (int64_t k = 0; k < n; ++k) {
        const int s = validate_rule(rules[k]);
        if (s != FW_OK) return set_status(s);
        if (first_ca < 0 && is_catch_all(rules[k])) first_ca = k;
    }
    fw_lindex *li = new (std::nothrow) fw_lindex();
    if (li == nullptr) return set_status(FW_ENOMEM);
    li->n = n;
    li->first_catch_all = first_ca;
    li->n_idx = (cfg.truncate != 2 && first_ca >= 0) ? first_ca + 1 : n;
    li->segments = segments;
    cudaGetDevice(&li->device);
    std::vector<uint8_t> class_of;
    std::vector<std::vector<int64_t>> lists;
    // a packet reads whole row words, 128 rules per uint4, at least one: a key
    // is taken only where it shortens those
    partition_lists(rules, li->n_idx, 128, class_of, lists, li->key_field, li->key_bits);
    li->n_classes = (int)lists.size();
    const int n_proto_classes = li->n_classes >> li->key_bits;
    std::vector<char> mixed((size_t)li->n_classes, 0);  // sub-list holds exact protocols of different values
    for (int c = 0; c < li->n_classes; ++c) {
        int first = -1;
        for (int64_t k : lists[c])
            if (!rules[k].proto_any) {
                if (first < 0) first = rules[k].proto;
                else if (rules[k].proto != first) mixed[c] = 1;
            }
        // the "other" class matches every protocol without a class: one exact rule is enough
        if ((c >> li->key_bits) == n_proto_classes - 1 && first >= 0) mixed[c] = 1;
    }
    std::vector<LiClassDev> hcls((size_t)li->n_classes);
    for (int c = 0; c < li->n_classes; ++c) {
        hcls[c].W = std::max<int64_t>(4, ((int64_t)lists[c].size() + 127) / 128 * 4);
        li->W = std::max(li->W, hcls[c].W);
    }

    cudaError_t e = cudaSuccess;
    std::vector<uint8_t> act((size_t)std::max<int64_t>(li->n_idx, 1), FW_DROP);
    for (int64_t k = 0; k < li->n_idx; ++k) act[k] = rules[k].action;
    e = dev_malloc(&li->d_class_of, 256);
    if (e == cudaSuccess) e = cudaMemcpy(li->d_class_of, class_of.data(), 256, cudaMemcpyHostToDevice);
    for (int c = 0; c < li->n_classes && e == cudaSuccess; ++c) {
        std::vector<int32_t> orig((size_t)hcls[c].W * 32, -1);
        for (size_t b = 0; b < lists[c].size(); ++b) orig[b] = (int32_t)lists[c][b];
        e = dev_malloc(&li->d_orig[c], orig.size() * sizeof(int32_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(li->d_orig[c], orig.data(), orig.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        fw_lindex_destroy(li);
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    if (e == cudaSuccess) e = dev_malloc(&li->d_action, act.size());
    if (e == cudaSuccess) e = cudaMemcpy(li->d_action, act.data(), act.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_malloc(&li->d_fallbacks, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(li->d_fallbacks, 0, sizeof(unsigned long long));
    uint32_t *d_rlo = nullptr, *d_rhi = nullptr;
    size_t nr = 1;
    for (const auto &L : lists) nr = std::max(nr, L.size());
    if (e == cudaSuccess) e = dev_malloc(&d_rlo, nr * 4);
    if (e == cudaSuccess) e = dev_malloc(&d_rhi, nr * 4);
    std::vector<uint32_t> rlo((size_t)std::max<int64_t>(li->n_idx, 1)), rhi(rlo.size()), clo(nr), chi(nr);
    for (int f = 0; f < kFields && e == cudaSuccess; ++f) {
        const int bits = kKeyBits[f];
        const int nseg = std::min(segments, 1 << std::min(bits, 16));
        int lg = 0;
        while ((1 << lg) < nseg) ++lg;
        li->shift[f] = bits - lg;
        std::vector<uint64_t> ends;
        ends.reserve(2 * li->n_idx + 1);
        ends.push_back(0);
        const uint64_t dom_end = uint64_t(1) << bits;
        for (int64_t k = 0; k < li->n_idx; ++k) {
            uint32_t lo, hi;
            field_interval(rules[k], f, lo, hi);
            rlo[k] = lo;
            rhi[k] = hi;
            ends.push_back(lo);
            if ((uint64_t)hi + 1 < dom_end) ends.push_back((uint64_t)hi + 1);
        }
        std::sort(ends.begin(), ends.end());
        ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
        std::vector<uint32_t> B(ends.begin(), ends.end());
        const int64_t M = (int64_t)B.size();
        li->M[f] = M;
        std::vector<float> A, Bc;
        std::vector<int32_t> E;
        fit_field(B, bits, nseg, li->shift[f], A, Bc, E, li->max_err[f]);
        e = dev_malloc(&li->d_bound[f], M * 4);
        if (e == cudaSuccess) e = dev_malloc(&li->d_model[f], nseg * sizeof(float4));
        if (e == cudaSuccess) e = cudaMemcpy(li->d_bound[f], B.data(), M * 4, cudaMemcpyHostToDevice);
        std::vector<float4> model((size_t)nseg);
        for (int s = 0; s < nseg; ++s) {
            float eb;
            std::memcpy(&eb, &E[s], sizeof(eb));
            model[s] = make_float4(A[s], Bc[s], eb, 0.0f);
        }
        if (e == cudaSuccess) e = cudaMemcpy(li->d_model[f], model.data(), nseg * sizeof(float4), cudaMemcpyHostToDevice);
        // rows of every class for this field; protocol rows only for a class whose
        // sub-list mixes exact protocols (elsewhere the class implies the protocol)
        for (int c = 0; c < li->n_classes && e == cudaSuccess; ++c) {
            if (f == kFields - 1 && !mixed[c]) continue;
            const int64_t nc = (int64_t)lists[c].size(), W = hcls[c].W;
            for (int64_t b = 0; b < nc; ++b) {
                clo[b] = rlo[lists[c][b]];
                chi[b] = rhi[lists[c][b]];
            }
            e = dev_malloc(&li->d_bits[c][f], (size_t)M * W * 4);
            if (e == cudaSuccess && nc > 0) e = cudaMemcpy(d_rlo, clo.data(), nc * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess && nc > 0) e = cudaMemcpy(d_rhi, chi.data(), nc * 4, cudaMemcpyHostToDevice);
            // short rows row by row, long rows quad-major (see LiClassDev)
            const int64_t Q = W / 4;
            const bool rm = li_row_major(W);
            if (e == cudaSuccess) {
                const int blocks = sm_count(li->device) * 8;
                k_li_build<<<blocks, 256>>>(li->d_bound[f], M, d_rlo, d_rhi, nc, Q, rm ? 1 : M, rm ? Q : 1,
                                            reinterpret_cast<uint4 *>(li->d_bits[c][f]));
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            hcls[c].bits[f] = reinterpret_cast<const uint4 *>(li->d_bits[c][f]);
            hcls[c].orig = li->d_orig[c];
            li->bitmap_bytes += (int64_t)M * W * 4;
        }
    }
    if (e == cudaSuccess) e = dev_malloc(&li->d_cls, hcls.size() * sizeof(LiClassDev));
    if (e == cudaSuccess)
        e = cudaMemcpy(li->d_cls, hcls.data(), hcls.size() * sizeof(LiClassDev), cudaMemcpyHostToDevice);
    cudaFree(d_rlo);
    cudaFree(d_rhi);
    if (e != cudaSuccess) {
        fw_lindex_destroy(li);
        cudaGetLastError();
        return set_status(cuda_status(e));
    }
    *out = li;
    return FW_OK;
}

extern "C" int fw_lindex_classify(const fw_lindex *li, const fw_headers *hdrs, int64_t n, int32_t *out_idx,
                                  uint8_t *out_act, void *stream) {
    if (li == nullptr || n < 0 || n > INT32_MAX) return set_status(FW_EINVAL);
    if (n == 0) return FW_OK;
    if (hdrs == nullptr || !hdrs->src || !hdrs->dst || !hdrs->sport || !hdrs->dport || !hdrs->proto || !out_idx ||
        !out_act)
        return set_status(FW_EINVAL);
    LiDev d;
    for (int f = 0; f < kFields; ++f) {
        d.f[f] = LiFieldDev{li->d_bound[f], li->d_model[f], (int32_t)li->M[f], li->shift[f]};
    }
    d.cls = li->d_cls;
    d.class_of = li->d_class_of;
    d.action = li->d_action;
    d.fallbacks = li->d_fallbacks;
    d.n_classes = li->n_classes;
    d.key_field = li->key_field;
    d.key_bits = li->key_bits;
    // the fields' interval starts in shared memory when they fit in 48 KB
    int64_t nb = 0;
    for (int f = 0; f < kFields; ++f) nb += li->M[f];
    const size_t sbytes = (size_t)nb * sizeof(uint32_t);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + 511) / 512, (int64_t)sm_count(li->device) * 4));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (sbytes <= 48 * 1024)
        k_li_classify<true><<<(unsigned)blocks, 512, sbytes, st>>>(d, hdrs->src, hdrs->dst, hdrs->sport, hdrs->dport,
                                                                    hdrs->proto, n, out_idx, out_act);
    else
        k_li_classify<false><<<(unsigned)blocks, 512, 0, st>>>(d, hdrs->src, hdrs->dst, hdrs->sport, hdrs->dport,
                                                                hdrs->proto, n, out_idx, out_act);
    return set_status(cuda_status(cudaGetLastError()));
}

extern "C" int fw_lindex_get_stats(fw_lindex *li, fw_lindex_stats *st) {
    if (li == nullptr || st == nullptr) return set_status(FW_EINVAL);
    std::memset(st, 0, sizeof(*st));
    st->rules = li->n;
    st->rules_indexed = li->n_idx;
    st->words_per_row = li->W;
    st->segments = li->segments;
    for (int f = 0; f < kFields; ++f) {
        st->intervals[f] = li->M[f];
        st->max_error[f] = li->max_err[f];
    }
    st->bitmap_bytes = li->bitmap_bytes;
    st->classes = li->n_classes;
    st->key_field = li->key_field;
    st->key_bits = li->key_bits;
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long fb = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&fb, li->d_fallbacks, sizeof(fb), cudaMemcpyDeviceToHost);
    st->fallbacks = (int64_t)fb;
    return set_status(cuda_status(e));
}
