// libmsc: kernels, fix-loop driver and the C ABI declared in include/msc.h.
//
// Device layout of one job (one original field f, N vertices):
//   f, f_hat, g, gprev    float[N]        resident for the job's lifetime; gprev holds the
//                                         pre-round value of the round's edited vertices
//   state                 uint8[N]        0..q_max quantised count, 0xF0 floor, 0xF1 exact
//   code_f, code_g        uint64[N]       packed gradient of the cells each anchor owns
//   low_f                 uint64[N]       (3D) f-lowest vertex slot of each triangle, tetrahedron
//   T/X/D bitsets         uint32[N/32]    targets, restores, dirty anchors (cleared per round)
//   T/X/D/E lists         uint32[N]       the same sets compacted; E = vertices a round changed
//   M/C bitsets           uint32[N/32]    anchors whose code / critical cells differ from f's
//   node words            16 bits per separatrix node (vertex, top cell, triangle, dead edge)
//   visited bitsets       N, 6N (3D) or 2N, 12N (3D) bits for the tier-3 walks
// The loop is incremental: after the initial dense gradient of g, a round re-evaluates only
// the anchors around edited vertices whose SoS order against a vertex within two edges
// changed, and targets only anchors whose critical cells differ from f's.  Large rounds run
// as captured graphs of per-step kernels, small ones in one persistent cooperative kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <unordered_map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/msc.h"
#include "msc_core.cuh"
#include "msc_dense.cuh"
#include "msc_runtime.h"

using namespace msc;

namespace {

thread_local std::string g_last_error;

msc_status fail(msc_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

}  // namespace

msc_status msc_rt::set_error(msc_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

namespace {

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (e_ == cudaErrorMemoryAllocation) return fail(MSC_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_)); \
            if (e_ == cudaErrorNoKernelImageForDevice || e_ == cudaErrorNoDevice ||            \
                e_ == cudaErrorInsufficientDriver)                                            \
                return fail(MSC_ERR_NO_DEVICE, "%s: %s", #call, cudaGetErrorString(e_));        \
            return fail(MSC_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                     \
    } while (0)

#define CKS(st)                                  \
    do {                                         \
        msc_status s_ = (st);                    \
        if (s_ != MSC_OK) return s_;             \
    } while (0)

constexpr int TPB = 256;

int sm_count()
{
    static const int sms = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 152;
    }();
    return sms;
}

// blocks of TPB threads of this kernel that fit on one SM at once (cached per kernel)
int occ_blocks(const void *kernel)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> cache;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &kv : cache)
        if (kv.first == kernel) return kv.second;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, TPB, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    cache.emplace_back(kernel, b);
    return b;
}

// whether the current device runs cooperative launches (the persistent round kernel)
bool coop_supported()
{
    static const bool ok = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev);
        return v != 0;
    }();
    return ok;
}

// grid for a grid-stride kernel over n threads' worth of work: at most one full wave of the
// blocks that can be resident at once, so no launch ends with a partly filled wave
int grid_occ(const void *kernel, unsigned long long n)
{
    unsigned long long b = (n + TPB - 1) / TPB;
    const unsigned long long cap = (unsigned long long)sm_count() * occ_blocks(kernel);
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// ------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------
#define GRID_STRIDE(i, n) for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < (n); \
                               i += (unsigned long long)gridDim.x * blockDim.x)

// Appends to a global list staged in shared memory: threads reserve slots with shared
// atomics and a block publishes its items with one global atomic per round (spilling
// straight to the list only if the stage is full), instead of one same-address global
// atomic per item.  Kernels using a stage run whole-block rounds of blockDim.x items.
template <int CAP> struct Stage {
    uint32_t buf[CAP];
    unsigned n;
    unsigned long long base;
};

template <int CAP> __device__ __forceinline__ void st_init(Stage<CAP> &s)
{
    if (threadIdx.x == 0) s.n = 0;
    __syncthreads();
}

template <int CAP> __device__ __forceinline__ void st_push(Stage<CAP> &s, uint32_t v, uint32_t *gl, unsigned long long *gn)
{
    const unsigned k = atomicAdd(&s.n, 1u);
    if (k < CAP) s.buf[k] = v;
    else gl[atomicAdd(gn, 1ull)] = v;
}

template <int CAP> __device__ __forceinline__ void st_flush(Stage<CAP> &s, uint32_t *gl, unsigned long long *gn)
{
    __syncthreads();
    const unsigned m = s.n < CAP ? s.n : CAP;
    if (threadIdx.x == 0 && m) s.base = atomicAdd(gn, (unsigned long long)m);
    __syncthreads();
    for (unsigned j = threadIdx.x; j < m; j += blockDim.x) gl[s.base + j] = s.buf[j];
    __syncthreads();
    if (threadIdx.x == 0) s.n = 0;
    __syncthreads();
}

// Appends to a global list staged per warp in shared memory: every lane of a converged warp
// offers at most one item per call, and the warp copies its stage to the list with one
// global atomic when the stage fills up and once at the end - no block-wide barrier, so the
// warps of a block never wait for one another.
template <int CAP> struct WarpStage {
    uint32_t buf[CAP];
    unsigned n;
};

template <int CAP> __device__ __forceinline__ void ws_flush(WarpStage<CAP> &s, uint32_t *gl, unsigned long long *gn)
{
    const unsigned lane = threadIdx.x & 31;
    __syncwarp();
    const unsigned m = s.n;
    if (m) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(gn, (unsigned long long)m);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (unsigned j = lane; j < m; j += 32) gl[base + j] = s.buf[j];
    }
    __syncwarp();
    if (lane == 0) s.n = 0;
    __syncwarp();
}

template <int CAP>
__device__ __forceinline__ void ws_push(WarpStage<CAP> &s, bool has, uint32_t v, uint32_t *gl, unsigned long long *gn)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    if (!mask) return;
    if (s.n + (unsigned)__popc(mask) > (unsigned)CAP) ws_flush(s, gl, gn);
    const unsigned pos = s.n + (unsigned)__popc(mask & ((1u << lane) - 1u));
    if (has) s.buf[pos] = v;
    __syncwarp();
    if (lane == 0) s.n += (unsigned)__popc(mask);
    __syncwarp();
}

// whole-block rounds over [0, n): every thread of a block runs the same number of rounds
#define BLOCK_ROUNDS(b, n) for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x; b < (n); \
                                b += (unsigned long long)gridDim.x * blockDim.x)

__global__ void k_count_nonfinite(const float *v, uint32_t n, unsigned long long *bad)
{
    unsigned long long local = 0;
    GRID_STRIDE(i, n) local += !isfinite(v[i]);
    if (local) atomicAdd(bad, local);
}

// dense gradient of a field; with ref != nullptr also list the anchors whose code differs
// (list, nlist) and those whose critical cells differ (clist, nclist; tier restricted)
// the anchors whose bit is set: each warp takes 32 consecutive words, compacts their set
// bits into shared memory (ascending anchor order, warp prefix sum of popcounts) and then
// runs f on them 32 at a time.  Needs blockDim.x == TPB.
template <class F>
__device__ __forceinline__ void for_each_set(const uint32_t *bits, uint32_t n, F &&f, unsigned long long *count = nullptr)
{
    __shared__ uint32_t q[TPB / 32][32 * 32];
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *mq = q[wib];
    const unsigned long long nw = (n + 31) / 32;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    for (unsigned long long w0 = warp * 32; w0 < nw; w0 += nwarps * 32) {
        uint32_t mine = w0 + lane < nw ? bits[w0 + lane] : 0u;
        const unsigned cnt = __popc(mine);
        unsigned pre = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= (unsigned)o) pre += y;
        }
        const unsigned total = __shfl_sync(0xffffffffu, pre, 31);
        if (total == 0) continue;
        if (count && lane == 0) atomicAdd(count, (unsigned long long)total);
        unsigned at = pre - cnt;
        const uint32_t base = (uint32_t)((w0 + lane) * 32);
        while (mine) {
            const int k = __ffs(mine) - 1;
            mine &= mine - 1;
            mq[at++] = base + (uint32_t)k;
        }
        __syncwarp();
        for (unsigned k = lane; k < total; k += 32) f(mq[k]);
        __syncwarp();
    }
}

// a no-op for the keep argument of cpass_listed
struct NoKeep {
    __device__ void operator()(uint32_t) const {}
};

// The C-pass over the listed blocks of the critical-difference bitset.  One warp per block
// compacts the block's set bits (anchors, ascending) into its row of q, then compacts the
// false cases of each group of 32 anchors (case_mask) into its row of cq, so that every lane
// applies one case (case_apply) instead of looping over its own anchor's cells while the
// other lanes wait.  Empty blocks have their summary bit cleared; non-empty blocks are handed
// to keep.  Needs blockDim.x == TPB.
constexpr int CASES_PER_ANCHOR = 26;
template <int D, bool GROUP, class K = NoKeep>
__device__ __forceinline__ void cpass_listed(const Ctx &c, uint16_t (*q)[32 * 32], uint16_t (*cq)[32 * CASES_PER_ANCHOR],
                                             const uint32_t *blk, unsigned long long nblk, unsigned long long *count,
                                             K &&keep = K{}, unsigned long long *next = nullptr)
{
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint16_t *mq = q[wib];   // anchors as offsets in their 1024-anchor block
    uint16_t *cw = cq[wib];
    const unsigned long long nw = (c.G.n + 31ull) / 32;
    // warps numbered across the blocks first (warp w of block b is b + w * blocks), so that a
    // few listed blocks spread over the SMs
    const unsigned long long warp = (unsigned long long)wib * gridDim.x + blockIdx.x;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    // with next: warps take blocks from a shared counter as they finish (blocks hold very
    // different numbers of cases); otherwise a fixed grid-stride share
    unsigned long long i = warp;
    for (;; i += nwarps) {
        if (next) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(next, 1ull);
            i = __shfl_sync(0xffffffffu, t, 0);
        }
        if (i >= nblk) break;
        const uint32_t b = blk[i];
        const unsigned long long w = (unsigned long long)b * 32 + lane;
        uint32_t mine = w < nw ? c.Cbits[w] : 0u;
        const unsigned cnt = __popc(mine);
        unsigned pre = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= (unsigned)o) pre += y;
        }
        const unsigned total = __shfl_sync(0xffffffffu, pre, 31);
        if (total == 0) {
            if (lane == 0) atomicAnd(c.Csum + (b >> 5), ~(1u << (b & 31)));
            continue;
        }
        if (lane == 0) {
            if (count) atomicAdd(count, (unsigned long long)total);
            keep(b);
        }
        unsigned at = pre - cnt;
        while (mine) {
            const int k = __ffs(mine) - 1;
            mine &= mine - 1;
            mq[at++] = (uint16_t)(lane * 32 + (unsigned)k);
        }
        __syncwarp();
        const uint32_t base = b * 1024u;
        for (unsigned k0 = 0; k0 < total; k0 += 32) {
            uint32_t m0 = 0;
            if (k0 + lane < total) {
                const uint32_t p = base + mq[k0 + lane];
                m0 = case_mask<D>(c, p, __ldg(c.code_f + p), c.code_g[p]);
            }
            // GROUP: the cases of these anchors one cell dimension at a time, so that the lanes
            // of a pass take the same branch of case_apply (mixed, a warp of a large C-pass ran
            // 9 of 32 lanes); a round of a few cases does better with one pass
            using Tb = Tab<D>;
            constexpr uint32_t GRP[4] = {1u, ((1u << Tb::NE) - 1u) << 1, ((1u << Tb::NT) - 1u) << (1 + Tb::NE),
                                         ((1u << Tb::NK) - 1u) << (1 + Tb::NE + Tb::NT)};
#pragma unroll
            for (int gi = 0; gi < (GROUP ? 4 : 1); gi++) {
                uint32_t m = GROUP ? m0 & GRP[gi] : m0;
                if (!__any_sync(0xffffffffu, m != 0)) continue;
                const unsigned nc = __popc(m);
                unsigned cpre = nc;
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, cpre, o);
                    if (lane >= (unsigned)o) cpre += y;
                }
                const unsigned ctot = __shfl_sync(0xffffffffu, cpre, 31);
                unsigned ca = cpre - nc;
                while (m) {
                    const int k = __ffs(m) - 1;
                    m &= m - 1;
                    cw[ca++] = (uint16_t)((lane << 5) | (unsigned)k);
                }
                __syncwarp();
                for (unsigned j = lane; j < ctot; j += 32) {
                    const unsigned e = cw[j];
                    case_apply<D>(c, base + mq[k0 + (e >> 5)], (int)(e & 31u));
                }
                __syncwarp();
            }
        }
    }
}

// list the blocks whose summary bit is set (appending to blk, count in *nblk); every warp
// of the grid takes 32 summary words at a time
__device__ __forceinline__ void list_blocks(const uint32_t *sum, unsigned long long nsum, uint32_t *blk,
                                            unsigned long long *nblk)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    for (unsigned long long w0 = warp * 32; w0 < nsum; w0 += nwarps * 32) {
        uint32_t mine = w0 + lane < nsum ? sum[w0 + lane] : 0u;
        const unsigned cnt = __popc(mine);
        unsigned pre = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= (unsigned)o) pre += y;
        }
        const unsigned total = __shfl_sync(0xffffffffu, pre, 31);
        if (total == 0) continue;
        unsigned long long at0 = 0;
        if (lane == 31) at0 = atomicAdd(nblk, (unsigned long long)total);
        at0 = __shfl_sync(0xffffffffu, at0, 31);
        unsigned long long at = at0 + pre - cnt;
        const uint32_t base = (uint32_t)((w0 + lane) * 32);
        while (mine) {
            const int k = __ffs(mine) - 1;
            mine &= mine - 1;
            blk[at++] = base + (uint32_t)k;
        }
    }
}

__host__ __device__ inline unsigned long long csum_words(uint32_t n) { return ((n + 31ull) / 32 + 1023) / 1024; }

// dense gradient of a field; with ref != nullptr also set the bitsets of anchors whose code
// differs (mbits) and whose critical cells differ (cbits, tier restricted)
template <int D>
__global__ void __launch_bounds__(TPB, 3) k_eval_dense(const float *v, Grid G, uint64_t *out, const uint64_t *ref,
                                                    uint32_t *mbits, uint32_t *cbits, uint32_t *csum, int tier)
{
    BLOCK_ROUNDS(b, G.n)
    {
        const unsigned long long p = b + threadIdx.x;
        bool m = false, cm = false;
        if (p < G.n) {
            const uint64_t code = anchor_code<D>(v, G, (uint32_t)p);
            out[p] = code;
            if (ref) {
                const uint64_t r = __ldg(ref + p);
                m = code != r;
                cm = m && crit_sig<D>(code, tier) != crit_sig<D>(r, tier);
            }
        }
        if (ref) {
            const uint32_t wm = __ballot_sync(0xffffffffu, m), wc = __ballot_sync(0xffffffffu, cm);
            if ((threadIdx.x & 31) == 0 && p < G.n) {
                mbits[p >> 5] = wm;
                cbits[p >> 5] = wc;
                if (wc) atomicOr(csum + (p >> 15), 1u << ((p >> 10) & 31));
            }
        }
    }
}

// Dense discrete gradient of a 3D field by z-marching tiles (msc_dense.cuh): grid
// (ceil(nx/32), ceil(ny/TY), ceil(nz/ZS)), 32 * TY threads.  With ref: also the bits of the
// anchors whose code differs from ref's (mbits) and whose critical cells differ (cbits,
// csum); mbits and cbits must be zero on entry (a warp's anchors need not start a word).
template <int TY, int ZS, int MINB>
__global__ void __launch_bounds__(32 * TY, MINB) k_eval_tile(const float *v, Grid G, uint64_t *out, const uint64_t *ref,
                                                            uint32_t *mbits, uint32_t *cbits, uint32_t *csum, int tier,
                                                            uint64_t *low, unsigned long long *seeds)
{
    using namespace dense;
    using T3 = Tab<3>;
    using TL = Tile<TY, ZS>;
    constexpr int TX = TL::TX, NT = TL::NT;
    unsigned long long nseed[3] = {0, 0, 0};
    constexpr int VX = TL::VX, VY = TL::VY, PX = TL::PX, PY = TL::PY, EX = TL::EX, EY = TL::EY, RX = TL::RX,
                  RY = TL::RY;
    __shared__ Smem<TL> S;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZS;
    const int zend = min(z0 + ZS, G.nz);
    const float INF = pos_inf();
    auto vs = [&](int z) { return (z - z0 + 2 * NVAL) % NVAL; };
    auto load_plane = [&](int z) {
        float(*P)[VX] = S.val[vs(z)];
        const bool zin = z >= 0 && z < G.nz;
        for (int i = tid; i < VX * VY; i += NT) {
            const int ly = i / VX, lx = i - ly * VX;
            const int x = x0 - 1 + lx, y = y0 - 1 + ly;
            P[ly][lx] = (zin && x >= 0 && x < G.nx && y >= 0 && y < G.ny) ? ld(v + vid(G, x, y, z)) : INF;
        }
    };
    load_plane(z0 - 1);
    load_plane(z0);
    const int nsteps = (zend - z0) + 3;
    for (int j = 0; j < nsteps; j++) {
        load_plane(z0 + j + 1);
        __syncthreads();
        // vertex pairs of plane zv (Sec. 4.2: the edge to the lowest lower neighbour)
        {
            const int zv = z0 + j;
            const float(*Pl[3])[VX] = {S.val[vs(zv - 1)], S.val[vs(zv)], S.val[vs(zv + 1)]};
            uint8_t(*Q)[PX] = S.vp[(zv - z0) % NVP];
            for (int i = tid; i < PX * PY; i += NT) {
                const int ly = i / PX, lx = i - ly * PX;
                float bv = INF;
                int bn = 15;
                static_for<14>([&](auto ic) {
                    constexpr int n = TabsC::D.vord[decltype(ic)::value];
                    constexpr int dx = TabC<3>::T.nb[n][0], dy = TabC<3>::T.nb[n][1], dz = TabC<3>::T.nb[n][2];
                    const float w = Pl[dz + 1][ly + 1 + dy][lx + 1 + dx];
                    if (w < bv) { bv = w; bn = n; }
                });
                const float wc = Pl[1][ly + 1][lx + 1];
                const bool below = bv < wc || (bv == wc && bn >= T3::NE);
                Q[ly][lx] = (uint8_t)(below ? bn : 15);
            }
        }
        __syncthreads();
        // edges of plane ze: paired down with the higher end, else up with the lowest cofacet
        // below both ends
        if (j >= 1) {
            const int ze = z0 + j - 1;
            const float(*Pl[4])[VX] = {S.val[vs(ze - 1)], S.val[vs(ze)], S.val[vs(ze + 1)], S.val[vs(ze + 2)]};
            const uint8_t(*Q[2])[PX] = {S.vp[(ze - z0) % NVP], S.vp[(ze + 1 - z0) % NVP]};
            uint32_t(*E)[EX] = S.ef[(ze - z0) % NEDG];
            for (int i = tid; i < EX * EY; i += NT) {
                const int ly = i / EX, lx = i - ly * EX;
                const float wa = Pl[1][ly + 1][lx + 1];
                const int vpa = Q[0][ly][lx];
                uint32_t fld = 0;
                static_for<7>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    constexpr int bx = TabsC::D.e_b[e][0], by = TabsC::D.e_b[e][1], bz = TabsC::D.e_b[e][2];
                    const float wb = Pl[1 + bz][ly + 1 + by][lx + 1 + bx];
                    const bool a_hi = wb < wa;
                    const bool down = a_hi ? (vpa == e) : ((int)Q[bz][ly + by][lx + bx] == T3::NE + e);
                    float bv = INF;
                    int bi = -1;
                    static_for<TabsC::D.e_nc[e]>([&](auto icc) {
                        constexpr int ci = decltype(icc)::value;
                        constexpr int dx = TabsC::D.e_c[e][ci][0], dy = TabsC::D.e_c[e][ci][1], dz = TabsC::D.e_c[e][ci][2];
                        const float w = Pl[1 + dz][ly + 1 + dy][lx + 1 + dx];
                        if (w < bv) { bv = w; bi = ci; }
                    });
                    constexpr unsigned mla = TabsC::D.e_lta[e], mlb = TabsC::D.e_ltb[e];
                    const bool lta = bi >= 0 && ((mla >> bi) & 1u);
                    const bool ltb = bi >= 0 && ((mlb >> bi) & 1u);
                    const bool below = (bv < wa || (bv == wa && lta)) && (bv < wb || (bv == wb && ltb));
                    const uint32_t f = down ? 1u : (below ? 2u + (uint32_t)bi : 0u);
                    fld |= f << (3 * e);
                });
                E[ly][lx] = fld;
            }
        }
        __syncthreads();
        // triangles of plane zt: paired down with the highest edge, else up with the lowest
        // tetrahedron candidate below all three vertices
        if (j >= 2) {
            const int zt = z0 + j - 2;
            const float(*Pl[4])[VX] = {S.val[vs(zt - 1)], S.val[vs(zt)], S.val[vs(zt + 1)], S.val[vs(zt + 2)]};
            const uint32_t(*E[2])[EX] = {S.ef[(zt - z0) % NEDG], S.ef[(zt + 1 - z0) % NEDG]};
            uint32_t(*R)[RX] = S.tf[(zt - z0) % NTRI];
            for (int i = tid; i < RX * RY; i += NT) {
                const int ly = i / RX, lx = i - ly * RX;
                uint32_t fld = 0;
                static_for<12>([&](auto tc) {
                    constexpr int t = decltype(tc)::value;
#define MSC_TV(s, k) TabsC::D.t_v[t][s][k]
                    const float w0 = Pl[1 + MSC_TV(0, 2)][ly + 1 + MSC_TV(0, 1)][lx + 1 + MSC_TV(0, 0)];
                    const float wA = Pl[1 + MSC_TV(1, 2)][ly + 1 + MSC_TV(1, 1)][lx + 1 + MSC_TV(1, 0)];
                    const float wB = Pl[1 + MSC_TV(2, 2)][ly + 1 + MSC_TV(2, 1)][lx + 1 + MSC_TV(2, 0)];
#undef MSC_TV
                    const bool la = w0 <= wA && w0 <= wB;
                    const bool lb = !la && wA <= wB;
                    uint32_t hf[3];
                    static_for<3>([&](auto jc) {
                        constexpr int s = decltype(jc)::value;
                        constexpr int hx = TabsC::D.t_he[t][s][0], hy = TabsC::D.t_he[t][s][1], hz = TabsC::D.t_he[t][s][2];
                        constexpr int hs = 3 * TabsC::D.t_het[t][s];
                        hf[s] = (E[hz][ly + hy][lx + hx] >> hs) & 7u;
                    });
                    constexpr unsigned hw0 = 2u + TabsC::D.t_hew[t][0], hw1 = 2u + TabsC::D.t_hew[t][1];
                    constexpr unsigned hw2 = 2u + TabsC::D.t_hew[t][2];
                    const bool down = la ? hf[0] == hw0 : (lb ? hf[1] == hw1 : hf[2] == hw2);
                    float bv = INF;
                    int bi = -1;
                    static_for<2>([&](auto icc) {
                        constexpr int ci = decltype(icc)::value;
                        constexpr int dx = TabsC::D.t_c[t][ci][0], dy = TabsC::D.t_c[t][ci][1], dz = TabsC::D.t_c[t][ci][2];
                        const float w = Pl[1 + dz][ly + 1 + dy][lx + 1 + dx];
                        if (w < bv) { bv = w; bi = ci; }
                    });
                    const float lv = la ? w0 : (lb ? wA : wB);
                    constexpr unsigned lt0 = TabsC::D.t_lt[t][0], lt1 = TabsC::D.t_lt[t][1], lt2 = TabsC::D.t_lt[t][2];
                    const unsigned ltm = la ? lt0 : (lb ? lt1 : lt2);
                    const bool below = bv < lv || (bv == lv && bi >= 0 && ((ltm >> bi) & 1u));
                    const uint32_t f = down ? 1u : (below ? 2u + (uint32_t)bi : 0u);
                    fld |= f << (2 * t);
                });
                R[ly][lx] = fld;
            }
        }
        __syncthreads();
        // codes of plane zk: tetrahedra (paired down iff their highest triangle chose them)
        // and the fields of every cell the anchor owns
        if (j >= 3) {
            const int zk = z0 + j - 3;
            const int lx = tid & 31, ly = tid >> 5;
            const int x = x0 + lx, y = y0 + ly;
            const bool valid = x < G.nx && y < G.ny;
            const float(*Pl[2])[VX] = {S.val[vs(zk)], S.val[vs(zk + 1)]};
            const uint32_t(*R[2])[RX] = {S.tf[(zk - z0) % NTRI], S.tf[(zk + 1 - z0) % NTRI]};
            uint64_t code = 0;
            unsigned long long p = 0;
            if (valid) {
                p = (unsigned long long)x + (unsigned long long)G.nx * ((unsigned long long)y + (unsigned long long)G.ny * zk);
                const unsigned cin = corner_mask<3>(G, x, y, zk);
                code = S.vp[(zk - z0) % NVP][ly][lx];
                const uint32_t efl = S.ef[(zk - z0) % NEDG][ly][lx];
                const uint32_t tfl = R[0][ly][lx];
                static_for<7>([&](auto ec) {
                    constexpr int e = decltype(ec)::value;
                    if ((cin >> (e + 1)) & 1u) code |= (uint64_t)((efl >> (3 * e)) & 7u) << (4 + 3 * e);
                });
                static_for<12>([&](auto tc) {
                    constexpr int t = decltype(tc)::value;
                    constexpr int top = TabC<3>::T.tB[t];
                    if ((cin >> top) & 1u) code |= (uint64_t)((tfl >> (2 * t)) & 3u) << (T3::TRI_BIT0 + 2 * t);
                });
                if ((cin >> 7) & 1u) {
                    static_for<6>([&](auto kc) {
                        constexpr int k = decltype(kc)::value;
                        float w[4];
                        static_for<4>([&](auto sc) {
                            constexpr int s = decltype(sc)::value;
                            constexpr int vx = TabsC::D.k_v[k][s][0], vy = TabsC::D.k_v[k][s][1], vz = TabsC::D.k_v[k][s][2];
                            w[s] = Pl[vz][ly + 1 + vy][lx + 1 + vx];
                        });
                        const bool l0 = w[0] <= w[1] && w[0] <= w[2] && w[0] <= w[3];
                        const bool l1 = !l0 && w[1] <= w[2] && w[1] <= w[3];
                        const bool l2 = !l0 && !l1 && w[2] <= w[3];
                        uint32_t ff[4];
                        static_for<4>([&](auto sc) {
                            constexpr int s = decltype(sc)::value;
                            constexpr int fx = TabsC::D.k_f[k][s][0], fy = TabsC::D.k_f[k][s][1], fz = TabsC::D.k_f[k][s][2];
                            constexpr int fs = 2 * TabsC::D.k_ft[k][s];
                            ff[s] = (R[fz][ly + fy][lx + fx] >> fs) & 3u;
                        });
                        constexpr unsigned fw0 = 2u + TabsC::D.k_fw[k][0], fw1 = 2u + TabsC::D.k_fw[k][1];
                        constexpr unsigned fw2 = 2u + TabsC::D.k_fw[k][2], fw3 = 2u + TabsC::D.k_fw[k][3];
                        const bool down = l0 ? ff[0] == fw0 : l1 ? ff[1] == fw1 : l2 ? ff[2] == fw2 : ff[3] == fw3;
                        code |= (uint64_t)down << (T3::TET_BIT0 + k);
                    });
                }
                out[p] = code;
                if (seeds)   // the separatrix seeds this anchor owns, counted from its code
                    for (int k = 0; k < 3; k++)
                        seeds_of_code<3>(code, G, (uint32_t)p, x, y, zk, k, [&](uint32_t) { nseed[k]++; });
                if (low) {
                    // lowest vertex slot of every triangle (bits 2t) and tetrahedron (bits 24 + 2k)
                    uint64_t lw = 0;
                    static_for<12>([&](auto tc) {
                        constexpr int t = decltype(tc)::value;
                        constexpr int az = TabsC::D.t_v[t][1][2], ay = TabsC::D.t_v[t][1][1], ax = TabsC::D.t_v[t][1][0];
                        constexpr int bz = TabsC::D.t_v[t][2][2], by = TabsC::D.t_v[t][2][1], bx = TabsC::D.t_v[t][2][0];
                        const float w0 = Pl[0][ly + 1][lx + 1];
                        const float wA = Pl[az][ly + 1 + ay][lx + 1 + ax];
                        const float wB = Pl[bz][ly + 1 + by][lx + 1 + bx];
                        const bool la = w0 <= wA && w0 <= wB, lb = !la && wA <= wB;
                        lw |= (uint64_t)(la ? 0 : (lb ? 1 : 2)) << (2 * t);
                    });
                    static_for<6>([&](auto kc) {
                        constexpr int k = decltype(kc)::value;
                        float w[4];
                        static_for<4>([&](auto sc) {
                            constexpr int s = decltype(sc)::value;
                            constexpr int vx = TabsC::D.k_v[k][s][0], vy = TabsC::D.k_v[k][s][1], vz = TabsC::D.k_v[k][s][2];
                            w[s] = Pl[vz][ly + 1 + vy][lx + 1 + vx];
                        });
                        const bool l0 = w[0] <= w[1] && w[0] <= w[2] && w[0] <= w[3];
                        const bool l1 = !l0 && w[1] <= w[2] && w[1] <= w[3];
                        const bool l2 = !l0 && !l1 && w[2] <= w[3];
                        lw |= (uint64_t)(l0 ? 0 : (l1 ? 1 : (l2 ? 2 : 3))) << (24 + 2 * k);
                    });
                    low[p] = lw;
                }
            }
            if (ref) {
                bool m = false, cm = false;
                if (valid) {
                    const uint64_t r = __ldg(ref + p);
                    m = code != r;
                    cm = m && crit_sig<3>(code, tier) != crit_sig<3>(r, tier);
                }
                const uint32_t wm = __ballot_sync(0xffffffffu, m), wc = __ballot_sync(0xffffffffu, cm);
                // lane k holds anchor p0 + k (lanes past the row end hold no bit)
                const unsigned long long p0 = __shfl_sync(0xffffffffu, p, 0);
                if (lx == 0 && (wm | wc)) {
                    const unsigned sh = (unsigned)(p0 & 31u);
                    const unsigned long long w0 = p0 >> 5;
                    if (wm) {
                        atomicOr(mbits + w0, wm << sh);
                        if (sh && (wm >> (32 - sh))) atomicOr(mbits + w0 + 1, wm >> (32 - sh));
                    }
                    if (wc) {
                        atomicOr(cbits + w0, wc << sh);
                        if (sh && (wc >> (32 - sh))) atomicOr(cbits + w0 + 1, wc >> (32 - sh));
                    }
                }
                if (cm) {
                    const uint32_t blk = (uint32_t)(p >> 10);
                    const unsigned peers = __match_any_sync(__activemask(), blk);
                    if ((unsigned)(__ffs(peers) - 1) == (unsigned)lx) atomicOr(csum + (blk >> 5), 1u << (blk & 31));
                }
            }
        }
        __syncthreads();
    }
    if (seeds) {
        // one atomic per warp and kind (every thread of the block reaches this point)
        for (int k = 0; k < 3; k++) {
            unsigned long long v = nseed[k];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(seeds + k, v);
        }
    }
}

// g = f_hat re-clamped into [f - xi, f + xi] (bounds rounded inward), every vertex unedited
// g's starting values; gprev starts equal to g (between rounds gprev[v] == g[v] for every v)
__global__ void k_init_g(const float *f, const float *fh, float *g, float *gprev, uint8_t *state, uint32_t n, float xi)
{
    GRID_STRIDE(i, n)
    {
        const float v = clamp_base(f[i], fh[i], xi);
        g[i] = v;
        gprev[i] = v;
        state[i] = 0;
    }
}

constexpr unsigned long long SMALL_ROUND = 8192;   // edited vertices below which rounds run small grids
constexpr unsigned long long CLUSTER_ROUND = 1024; // and below which they run in one thread-block cluster

// a round kernel of a captured round graph does nothing once the phase is over (halt) or
// the rounds have become small (leave)
__device__ __forceinline__ bool round_off(const LoopState *ls) { return ls->halt || ls->leave; }

// ---- one edit round as a chain of kernels that read the device loop state (ls): any
// kernel of a round whose phase is over (ls->halt) or whose rounds have become small
// (ls->leave) does nothing, so rounds can be queued back to back (a captured graph of
// several rounds) and the host looks only at their end.

// case tallies of the persistent round kernel's C-pass, kept per block in shared memory and
// published once (k_ctargets keeps them per warp)
struct BlockTally {
    unsigned long long v[2];
};

__device__ __forceinline__ void tally_begin(BlockTally &t, Ctx &cc)
{
    if (threadIdx.x < 2) t.v[threadIdx.x] = 0;
    __syncthreads();
    cc.tally = t.v;
}

__device__ __forceinline__ void tally_end(BlockTally &t, const Ctx &c)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        if (t.v[0]) atomicAdd(&c.cnt->ncase, t.v[0]);
        if (t.v[1]) atomicAdd(&c.cnt->nlive, t.v[1]);
    }
}

template <int D> __global__ void __launch_bounds__(TPB, 4) k_ctargets(Ctx c)
{
    if (round_off(c.ls)) return;
    __shared__ unsigned long long wt[TPB / 32][2];   // per-warp case tallies
    __shared__ uint16_t q[TPB / 32][32 * 32];
    __shared__ uint16_t cq[TPB / 32][32 * CASES_PER_ANCHOR];
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane < 2) wt[wib][lane] = 0;
    __syncwarp();
    Ctx cc = c;
    cc.tally = wt[wib];
    cpass_listed<D, true>(cc, q, cq, c.Cblk, c.ls->nblk, &c.ls->cpass_items, NoKeep{}, &c.cnt->wnext);
    __syncwarp();
    if (lane == 0) {
        if (wt[wib][0]) atomicAdd(&c.cnt->ncase, wt[wib][0]);
        if (wt[wib][1]) atomicAdd(&c.cnt->nlive, wt[wib][1]);
    }
}

// the T list of a round whose C-pass only set T bits (mark_only): one warp per 32 bitset
// words, one atomic per warp for its slots and one for its sum of vertex ids
__global__ void k_tlist(Ctx c)
{
    if (round_off(c.ls)) return;
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long nw = (c.G.n + 31ull) / 32;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    for (unsigned long long w0 = warp * 32; w0 < nw; w0 += nwarps * 32) {
        uint32_t mine = w0 + lane < nw ? c.Tbits[w0 + lane] : 0u;
        const unsigned cnt = __popc(mine);
        unsigned pre = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= (unsigned)o) pre += y;
        }
        const unsigned total = __shfl_sync(0xffffffffu, pre, 31);
        if (total == 0) continue;
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&c.cnt->nT, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 31);
        unsigned long long at = base + pre - cnt, sum = 0;
        const uint32_t v0 = (uint32_t)((w0 + lane) * 32);
        while (mine) {
            const int k = __ffs(mine) - 1;
            mine &= mine - 1;
            c.Tlist[at++] = v0 + (uint32_t)k;
            sum += v0 + (uint32_t)k;
        }
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) atomicAdd(&c.cnt->sumT, sum);
    }
}

// after a targeting pass (kind 0 C, 1 S): stop the phase when there is no false case, stop
// with a status on a stall or at max_iters.  iters: the loop's round count when the pass
// began.
__device__ __forceinline__ bool round_stop(const LoopState *ls, const Counters *k, unsigned iters, int &status)
{
    status = 0;
    if (k->ncase == 0) return true;
    if (!ls->exact_fallback && k->nlive == 0) { status = MSC_ERR_STALLED; return true; }
    if (iters >= ls->max_iters) { status = MSC_ERR_NOT_CONVERGED; return true; }
    return false;
}

// record the decision (one thread): halt with the status, or count and trace the round
__device__ void round_record(const Ctx &c, const Counters *k, int kind, bool stop, int status)
{
    LoopState *ls = c.ls;
    ls->cases += k->ncase;
    if (stop) {
        ls->halt = 1;
        if (status) ls->status = status;
        return;
    }
    if (c.trace && ls->ntrace < ls->trace_cap) {
        int64_t *r = c.trace + 6 * (size_t)ls->ntrace;
        r[0] = kind; r[1] = (int64_t)k->nT; r[2] = (int64_t)k->nX; r[3] = (int64_t)k->sumT; r[4] = (int64_t)k->sumX;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        r[5] = (int64_t)t;
    }
    ls->ntrace++;
    ls->iters++;
    if (kind) ls->n_s++; else ls->n_c++;
    if (k->nX) ls->n_fb++;
    ls->edit_items += k->nT + k->nX;
    ls->last_items = k->nT + k->nX;
}

__global__ void k_decide(Ctx c, int kind)
{
    if (threadIdx.x || blockIdx.x) return;
    LoopState *ls = c.ls;
    if (round_off(ls)) return;
    ls->nblk = 0;          // the C-pass has read the block list; the round's end lists it anew
    int status;
    const bool stop = round_stop(ls, c.cnt, ls->iters, status);
    round_record(c, c.cnt, kind, stop, status);
}


// one thread per edit item: save the pre-round value, apply Eq. 2 (or the restore), and
// list the vertices whose value changed
template <int D> __global__ void k_edit(Ctx c)
{
    if (round_off(c.ls)) return;
    __shared__ WarpStage<256> se[TPB / 32];
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (lane == 0) se[wib].n = 0;
    __syncwarp();
    const unsigned long long nX = c.cnt->nX, items = nX + c.cnt->nT;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    for (unsigned long long b = warp * 32; b < items; b += nwarps * 32) {
        const unsigned long long i = b + lane;
        uint32_t v = 0;
        bool changed = false;
        if (i < items && edit_prepare(c, (uint32_t)i, (uint32_t)nX, v)) {
            edit_apply(c, (uint32_t)i, (uint32_t)nX, v);
            changed = true;
        }
        ws_push(se[wib], changed, v, c.Elist, &c.cnt->nE);
    }
    ws_flush(se[wib], c.Elist, &c.cnt->nE);
}

// what one lane of a warp handles of a changed vertex, held in registers for a whole kernel:
// ring offsets lane and lane + 32 (the vertices whose order against it a rule compares) and
// window row `lane`
struct LaneGeom {
    int rg[2][3];        // ring offsets lane and lane + 32
    bool ron[2];
    uint64_t rwin[2];    // their window masks (RingWin)
    int wg[2][3];        // window offsets lane and lane + 32
    bool won[2];
};
template <int D> __device__ __forceinline__ LaneGeom lane_geom(unsigned lane)
{
    const Tab<D> &T = rt_tab<D>();
    const RingWin<D> &RW = rt_ring_win<D>();
    LaneGeom g;
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int j = (int)lane + 32 * r;
        g.ron[r] = j < T.nring;
        for (int k = 0; k < 3; k++) g.rg[r][k] = g.ron[r] ? T.ring[j][k] : 0;
        g.rwin[r] = g.ron[r] ? RW.m[j] : 0ull;
        g.won[r] = j < T.nwin;
        for (int k = 0; k < 3; k++) g.wg[r][k] = g.won[r] ? T.win[j][k] : 0;
    }
    return g;
}

// The order-change test of an edited vertex v (lanes as parts, ring offsets from LaneGeom):
// the window positions of v whose anchors a flipped pair (v, u) can change, OR-ed over the
// warp (every lane gets the same mask).  A neighbour's value before the round is gprev's:
// between rounds gprev equals g everywhere, and a round saves the pre-round value of each
// vertex it edits there.
template <int D>
__device__ __forceinline__ uint64_t ring_window_mask(const Ctx &c, uint32_t v, int x, int y, int z, const LaneGeom &g)
{
    const float ov = c.gprev[v], nv = c.g[v];
    uint64_t m = 0;
#pragma unroll
    for (int r = 0; r < 2; r++) {
        if (!g.ron[r]) continue;
        const int ux = x + g.rg[r][0], uy = y + g.rg[r][1], uz = z + g.rg[r][2];
        if (!inside(c.G, ux, uy, uz)) continue;
        const uint32_t u = vid(c.G, ux, uy, uz);
        const float nu = c.g[u], ou = c.gprev[u];
        if (sos_lt(ov, v, ou, u) != sos_lt(nv, v, nu, u)) m |= g.rwin[r];
    }
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)m), hi = __reduce_or_sync(0xffffffffu, (unsigned)(m >> 32));
    return ((uint64_t)hi << 32) | lo;
}

// the anchor at window position lane + 32 r of v, if the mask holds it and it is inside the
// domain; false otherwise
__device__ __forceinline__ bool window_anchor(const Ctx &c, const LaneGeom &g, uint64_t mask, int r, int x, int y, int z,
                                              uint32_t &p)
{
    const int j = (int)(threadIdx.x & 31) + 32 * r;
    if (!g.won[r] || !((mask >> j) & 1ull)) return false;
    const int px = x - g.wg[r][0], py = y - g.wg[r][1], pz = z - g.wg[r][2];
    if (!inside(c.G, px, py, pz)) return false;
    p = vid(c.G, px, py, pz);
    return true;
}

// one warp per changed vertex: the lanes test its order against the vertices within two
// edges and mark dirty the anchors of its window that hold both ends of a flipped pair;
// without a flip no code can change and nothing is marked.  (One thread per vertex loads
// less in the largest rounds, but runs the ~60 ring checks of a vertex one after another in
// the middle-sized ones, and lists the dirty anchors in an order that costs the refresh more
// than it saves.)
template <int D> __global__ void k_mark(Ctx c)
{
    if (round_off(c.ls)) return;
    __shared__ WarpStage<512> sd[TPB / 32];
    __shared__ LaneGeom lgs[32];
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (threadIdx.x < 32) lgs[lane] = lane_geom<D>(lane);
    if (lane == 0) sd[wib].n = 0;
    __syncthreads();
    const unsigned long long items = c.cnt->nE;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    for (unsigned long long i = warp; i < items; i += nwarps) {
        const uint32_t v = c.Elist[i];
        int x, y, z;
        coords(c.G, v, x, y, z);
        const uint64_t mask = ring_window_mask<D>(c, v, x, y, z, lgs[lane]);
        if (!mask) continue;                     // the same in every lane
#pragma unroll
        for (int r = 0; r < 2; r++) {            // the window has at most 64 anchors
            uint32_t p = 0;
            const bool has = window_anchor(c, lgs[lane], mask, r, x, y, z, p) && !test_and_set(c.Dbits, p);
            ws_push(sd[wib], has, p, c.Dlist, &c.cnt->nD);
        }
    }
    ws_flush(sd[wib], c.Dlist, &c.cnt->nD);
}

template <int D> __global__ void __launch_bounds__(TPB, 3) k_refresh(Ctx c)
{
    if (round_off(c.ls)) return;
    const unsigned long long n = c.cnt->nD;
    GRID_STRIDE(i, n) refresh_anchor<D>(c, c.Dlist[i]);
}

// mismatch bits of a re-evaluated anchor p with code cg: M (code differs from f's) and C
// (critical cells differ), and the C summary bit of p's 1024-anchor block.  Returns
// whether this call set that summary bit.
template <int D> __device__ __forceinline__ bool rebuild_anchor(const Ctx &c, uint32_t p, uint64_t cg)
{
    const uint64_t cf = __ldg(c.code_f + p);
    const bool m = cf != cg, cm = m && crit_sig<D>(cf, c.tier) != crit_sig<D>(cg, c.tier);
    const uint32_t bit = 1u << (p & 31);
    if (m) atomicOr(c.Mbits + (p >> 5), bit); else atomicAnd(c.Mbits + (p >> 5), ~bit);
    if (!cm) {
        atomicAnd(c.Cbits + (p >> 5), ~bit);
        return false;
    }
    atomicOr(c.Cbits + (p >> 5), bit);
    const uint32_t sb = 1u << ((p >> 10) & 31);
    if (c.Csum[p >> 15] & sb) return false;
    return !(atomicOr(c.Csum + (p >> 15), sb) & sb);
}

// mismatch bitsets after a round: only re-evaluated (dirty) anchors can change membership.
// A refreshed anchor also joins the separatrix dirty set (a bit, set without waiting for
// the old value; the S-pass lists the set bits once, k_sd_list).
template <int D> __global__ void k_rebuild(Ctx c)
{
    if (round_off(c.ls)) return;
    LoopState *ls = c.ls;
    const unsigned long long d = c.cnt->nD;
    const int track = ls->track_dirty;
    GRID_STRIDE(i, d)
    {
        const uint32_t p = c.Dlist[i];
        if (track) atomicOr(c.sDbits + (p >> 5), 1u << (p & 31));
        rebuild_anchor<D>(c, p, c.code_g[p]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ls->refresh_items, d);
}

// end of a round's edits: clear the round's sets through their lists (and bring gprev back
// to g at the round's items: between rounds gprev equals g everywhere, so the order-change
// test reads a neighbour's pre-round value from gprev without asking whether it moved), and
// list the blocks of the critical-difference bitset that the next C-pass visits
__device__ __forceinline__ void clear_item(const Ctx &c, unsigned long long i, unsigned long long nT, unsigned long long nX)
{
    if (i < nT) {
        const uint32_t v = c.Tlist[i];
        c.Tbits[v >> 5] = 0;
        c.gprev[v] = c.g[v];
    } else if (i < nT + nX) {
        const uint32_t v = c.Xlist[i - nT];
        c.Xbits[v >> 5] = 0;
        c.gprev[v] = c.g[v];
    } else {
        c.Dbits[c.Dlist[i - nT - nX] >> 5] = 0;
    }
}

__global__ void k_clear(Ctx c)
{
    if (round_off(c.ls)) return;
    const unsigned long long nT = c.cnt->nT, nX = c.cnt->nX, nD = c.cnt->nD;
    GRID_STRIDE(i, nT + nX + nD) clear_item(c, i, nT, nX);
    list_blocks(c.Csum, csum_words(c.G.n), c.Cblk, &c.ls->nblk);
}

__global__ void k_list_blocks(Ctx c) { list_blocks(c.Csum, csum_words(c.G.n), c.Cblk, &c.ls->nblk); }

// end of a round: zero the round's counters
__global__ void k_end(Ctx c)
{
    if (threadIdx.x || blockIdx.x || round_off(c.ls)) return;
    memset(c.cnt, 0, sizeof(Counters));
    if (c.ls->rounds_kernel && c.ls->last_items < c.ls->small_round) c.ls->leave = 1;
}

__global__ void k_set_leave(LoopState *ls, int v) { ls->leave = v; }

__global__ void k_set_halt(LoopState *ls, int v) { ls->halt = v; }
__global__ void k_set_track(LoopState *ls, int v) { ls->track_dirty = v; }

// ---- persistent C-pass rounds.  Rounds that edit few vertices cost mostly the gaps between
// their kernels, so the rounds after the first large ones run in one cooperative launch (all
// blocks resident), their phases separated by grid barriers:
//   P1 targets (C-pass) | P2 decision + edits | P3 order changes -> dirty anchors |
//   P4 refresh + mismatch bits + clearing the round's sets
// The C-pass visits a list of 1024-anchor blocks kept in two buffers: the blocks P1 finds
// non-empty and the blocks whose summary bit P4 newly sets form the next round's list.  The
// round counters alternate between two Counters by round parity, so a round's counters are
// zeroed while the round after it runs.  Data written by other blocks is read with plain
// (coherent) loads after a barrier, never through the read-only path.
constexpr int ROUND_STAGE = 4096;                          // dirty-anchor stage entries
constexpr unsigned long long BAR_TIMEOUT_NS = 2000000000ull;   // 2 s
constexpr unsigned BAR_SPIN_CAP = 1u << 28;

struct GridBarrier {
    unsigned arrive, gen;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch.  The wait is bounded: a block that waits longer
// than BAR_TIMEOUT_NS records MSC_ERR_DEVICE_TIMEOUT in the loop state and returns false, and
// so does every block that passes a barrier after that, so the kernel always ends.
__device__ bool grid_sync(GridBarrier *gb, LoopState *ls, unsigned long long timeout_ns = BAR_TIMEOUT_NS)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &gb->gen;
        const unsigned g0 = *gen;
        __threadfence();
        int good = 1;
        if (atomicAdd(&gb->arrive, 1u) == gridDim.x - 1) {
            atomicExch(&gb->arrive, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            unsigned spins = 0;
            while (*gen == g0) {
                if (++spins >= BAR_SPIN_CAP || ((spins & 63u) == 0 && global_ns() - t0 > timeout_ns)) {
                    good = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        if (!good) {
            atomicExch(&ls->status, (int)MSC_ERR_DEVICE_TIMEOUT);
            atomicExch(&ls->halt, 1);
        }
        if (((volatile int *)&ls->status)[0] == (int)MSC_ERR_DEVICE_TIMEOUT) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Barrier between the phases of a round.  Full-grid form (cooperative launch): the bounded
// grid barrier above.  Cluster form (the whole grid is one thread-block cluster): the
// hardware cluster barrier with release/acquire at cluster scope, then a fence so that the
// data other blocks wrote is read fresh, as after the grid barrier.  It waits for every
// thread of every block of the cluster; every block reaches it the same number of times,
// because each return below is taken by all threads alike (after a barrier, from the same
// counters).
template <bool CL> __device__ __forceinline__ bool round_sync(GridBarrier *gb, LoopState *ls)
{
    if constexpr (CL) {
        asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
        __threadfence();
        return true;
    } else {
        return grid_sync(gb, ls);
    }
}

template <int D, bool CL>
__global__ void __launch_bounds__(TPB, 2) k_rounds(Ctx c, GridBarrier *gb, Counters *cnt2, uint32_t *blk2, unsigned max_rounds,
                                                unsigned long long leave_items, unsigned long long leave_below,
                                                unsigned long long blk_limit)
{
    __shared__ union {
        uint16_t q[TPB / 32][32 * 32];   // P1: compacted anchors of a block, per warp
        Stage<ROUND_STAGE> sd;           // P3: dirty anchors
    } u;
    __shared__ uint16_t cq[TPB / 32][32 * CASES_PER_ANCHOR];   // P1: compacted false cases
    __shared__ BlockTally tally;
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    __shared__ LaneGeom lgs[32];         // the same for every warp: kept in shared memory, where
    if (threadIdx.x < 32) lgs[lane] = lane_geom<D>(lane);   // registers are scarce here
    __syncthreads();
    const LaneGeom &lg = lgs[lane];
    LoopState *ls = c.ls;
    uint32_t *const lists[2] = {c.Cblk, blk2};
    const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long gtid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long sgtid = (unsigned long long)threadIdx.x * gridDim.x + blockIdx.x;   // spread order
    unsigned long long tph = gtid == 0 ? global_ns() : 0;
    auto phase_end = [&](int ph) {   // block 0, thread 0: time since the last barrier
        if (gtid != 0) return;
        const unsigned long long t = global_ns();
        ls->phase_ns[ph] += t - tph;
        tph = t;
    };
    for (unsigned r = 0; r < max_rounds; r++) {
        const int cur = (int)(r & 1u), nxt = cur ^ 1;
        Counters *K = cnt2 + cur;
        Ctx cc = c;
        cc.cnt = K;
        const unsigned iters = ls->iters;        // block 0 advances it only after barrier 1
        // P1: false cases of the listed blocks; non-empty blocks stay listed
        if (gtid == 0) memset(cnt2 + nxt, 0, sizeof(Counters));
        tally_begin(tally, cc);
        {
            // The C-pass reads the pre-round values (gprev equals g between rounds) and edits
            // each target it lists at once into g (fuse_target), unless this round would be
            // past max_iters.  No separate edit phase: a round that stops edits nothing (no
            // case, or every target stuck at the floor or restored), and the rare restores of
            // the exact fallback are applied after the barrier, overriding a target's step.
            Ctx cp = cc;
            cp.g = c.gprev;
            cp.fuse_g = iters < ls->max_iters ? c.g : nullptr;
            uint32_t *nl = lists[nxt];
            unsigned long long *nn = &ls->nbl[nxt];
            cpass_listed<D, false>(cp, u.q, cq, lists[cur], ls->nbl[cur], &ls->cpass_items,
                                   [&](uint32_t b) { nl[atomicAdd(nn, 1ull)] = b; });
        }
        tally_end(tally, cc);
        if (!round_sync<CL>(gb, ls)) return;
        phase_end(0);
        // P2: the decision, taken alike by every thread from the finished counters (block 0
        // records it); then the restores, if any (dealt round-robin over the blocks)
        int status;
        const bool stop = round_stop(ls, K, iters, status);
        const unsigned long long nX = K->nX, items = nX + K->nT;
        if (gtid == 0) round_record(cc, K, 0, stop, status);
        if (stop) return;
        if (nX) {
            for (unsigned long long i = sgtid; i < nX; i += nthreads) {
                const uint32_t v = c.Xlist[i];
                if (c.state[v] != ST_EXACT) {
                    c.g[v] = ld(c.f + v);
                    c.state[v] = ST_EXACT;
                    c.Elist[list_slot(&K->nE)] = v;
                }
            }
            if (!round_sync<CL>(gb, ls)) return;
        }
        phase_end(1);
        // P3: edited vertices whose order changed mark their windows dirty
        st_init(u.sd);
        const unsigned long long nE = K->nE;
        for (unsigned long long k0 = 0; k0 < nE; k0 += (unsigned long long)gridDim.x * wpb) {
            const unsigned long long i = k0 + (unsigned long long)wib * gridDim.x + blockIdx.x;
            if (i < nE) {
                const uint32_t v = c.Elist[i];
                if (lane == 0) state_after(cc, v);   // the state of a target edited in P1
                int x, y, z;
                coords(c.G, v, x, y, z);
                const uint64_t mask = ring_window_mask<D>(cc, v, x, y, z, lg);
                if (mask)
#pragma unroll
                    for (int r = 0; r < 2; r++) {
                        uint32_t p;
                        if (window_anchor(cc, lg, mask, r, x, y, z, p) && !test_and_set(c.Dbits, p))
                            st_push(u.sd, p, c.Dlist, &K->nD);
                    }
            }
            st_flush(u.sd, c.Dlist, &K->nD);
        }
        if (!round_sync<CL>(gb, ls)) return;
        phase_end(2);
        // P4: new codes and mismatch bits of the dirty anchors; clear the round's sets
        const unsigned long long nD = K->nD, nT = K->nT;
        const int track = ls->track_dirty;
        for (unsigned long long i = sgtid; i < nD; i += nthreads) {
            const uint32_t p = c.Dlist[i];
            const uint64_t cg = anchor_code<D, false>(c.g, c.G, p);
            c.code_g[p] = cg;
            if (track) atomicOr(c.sDbits + (p >> 5), 1u << (p & 31));
            if (rebuild_anchor<D>(cc, p, cg)) lists[nxt][atomicAdd(&ls->nbl[nxt], 1ull)] = p >> 10;
        }
        for (unsigned long long i = sgtid; i < nT + nX + nD; i += nthreads) clear_item(c, i, nT, nX);
        if (gtid == 0) {
            atomicAdd(&ls->refresh_items, nD);
            ls->nbl[cur] = 0;                    // list cur was read in P1; it is the next "next"
        }
        if (!round_sync<CL>(gb, ls)) return;
        phase_end(3);
        // a large round: the next rounds run full grids; a tiny one in the full-grid form: the
        // next rounds run in one cluster.  The cluster form also leaves, and the full-grid form
        // keeps the rounds, while the next round's C-pass lists more blocks than the cluster has
        // warps to share them (the list is final after the barrier above, the same for all).
        const bool few_blocks = ls->nbl[nxt] <= blk_limit;
        if (items >= leave_items || (CL && !few_blocks) || (items < leave_below && few_blocks)) return;
    }
}

// entry state of k_rounds: the C-block list of the round graphs is list 0
__global__ void k_rounds_enter(LoopState *ls, GridBarrier *gb)
{
    ls->leave = 0;
    ls->nbl[0] = ls->nblk;
    ls->nbl[1] = 0;
    gb->arrive = 0;
}

// after k_rounds: list the C blocks again for the round graphs and the S-pass edit round
__global__ void k_rounds_leave(LoopState *ls) { ls->nblk = 0; }

// self-test of the bounded grid barrier: block 0 waits at a barrier that the other blocks
// never reach (they return at once), so its wait must give up after timeout_ns
__global__ void k_barrier_selftest(GridBarrier *gb, LoopState *ls, unsigned long long timeout_ns)
{
    if (blockIdx.x != 0) return;
    grid_sync(gb, ls, timeout_ns);
}

template <int D> __global__ void k_desc(Ctx c, const uint32_t *seeds, uint32_t n)
{
    GRID_STRIDE(i, n) desc_walk<D>(c, seeds[i]);
}

template <int D> __global__ void k_asc(Ctx c, const uint32_t *seeds, uint32_t n)
{
    GRID_STRIDE(i, n) asc_walk<D>(c, seeds[i]);
}

__global__ void k_ss_seed(Ctx c, const uint32_t *seeds, uint32_t n)
{
    GRID_STRIDE(i, n) ss_walk(c, seeds[i], 0xFFFFFFFFu, true);
}

__global__ void k_ss_spill(Ctx c, const uint32_t *items, uint32_t n)
{
    GRID_STRIDE(i, n) ss_walk(c, items[2 * i], items[2 * i + 1], false);
}

// verification of saddle-saddle connectors: one backward step from each listed triangle
__global__ void k_ss_back(Ctx c, const uint32_t *in, uint32_t n, uint32_t *out, unsigned long long *nout, uint32_t cap)
{
    GRID_STRIDE(i, n) ss_back_step(c, in[i], out, nout, cap);
}

// 2-saddles whose connectors reach a troublemaker, counted into *n
__global__ void k_ss_count(Ctx c, const uint32_t *seeds, uint32_t n, unsigned long long *cnt)
{
    GRID_STRIDE(i, n)
    {
        const uint32_t t = seeds[i];
        count_add(cnt, (c.ss_bad[t >> 5] >> (t & 31)) & 1u);
    }
}

template <int D> __global__ void __launch_bounds__(TPB) k_node_init(Ctx c)
{
    GRID_STRIDE(p, c.G.n) node_bits<D>(c, (uint32_t)p, true);
}

// two walk slots per lane at 6 blocks per SM (512^3 first build: 4 slots at 4 blocks 25.5 ms,
// 2 at 6: 24.4 ms, 4 at 3: 27.0, 4 or 8 at 2: 31.0)
template <int D> __global__ void __launch_bounds__(TPB, 6) k_node_seed(Ctx c, int kind, const uint32_t *seeds, uint32_t n)
{
    path_seed_walks<D, 2>(c, kind, seeds, n, (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5,
                          (gridDim.x * (unsigned long long)blockDim.x) >> 5);
}

// the first build's saddle-saddle propagation (3D): per-warp stacks in shared memory.  It
// runs at most SS_BLOCKS_PER_SM blocks per SM: more warps walking at once contend for L1 and
// L2 and finish later (kolmogorov3d 512^3: 8 blocks per SM 22 ms, 6: 19.5 ms, 4: 19.6 ms,
// 3: 23 ms).
constexpr int SS_WARP_STACK = 384;
constexpr int SS_BLOCKS_PER_SM = 6;
__global__ void k_node_seed_ss(Ctx c, const uint32_t *seeds, uint32_t n)
{
    __shared__ uint32_t stk[TPB / 32][SS_WARP_STACK];
    __shared__ int8_t sdl[TPB / 32][SS_WARP_STACK];
    const unsigned wib = threadIdx.x >> 5;
    tri_seed_walks(c, seeds, n, stk[wib], sdl[wib], (int)c.ss_stack_cap);
}

template <int D> __global__ void k_node_update(Ctx c, const unsigned long long *nSD)
{
    const unsigned long long n = *nSD;
    GRID_STRIDE(i, n) node_bits<D>(c, c.sDlist[i], false);
}

// (triangle, delta) items of the spill queue: the converged per-warp stack walk of the first
// build, fed with items instead of seeds
__global__ void k_tri_spill(Ctx c, const uint32_t *items, uint32_t n)
{
    __shared__ uint32_t stk[TPB / 32][SS_WARP_STACK];
    __shared__ int8_t sdl[TPB / 32][SS_WARP_STACK];
    const unsigned wib = threadIdx.x >> 5;
    tri_seed_walks<true>(c, items, n, stk[wib], sdl[wib], (int)c.ss_stack_cap);
}

// Troublemakers at the mismatched anchors.  A warp compacts the set bits of 32 words of the
// mismatch bitset, then takes its anchors 32 at a time and their differing pair fields one
// kind at a time (vertex, facet, edge), so that the lanes of a pass run the same branch of
// node_target_item (per anchor, a warp ran ~5 of 32 lanes).
template <int D> __global__ void k_node_targets(Ctx c)
{
    __shared__ BlockTally tally;
    __shared__ uint32_t aq[TPB / 32][32 * 32];
    __shared__ uint16_t fq[TPB / 32][32 * 16];   // one kind's fields of 32 anchors (at most 12 each)
    Ctx cc = c;
    tally_begin(tally, cc);
    constexpr int NFAC = D == 3 ? Tab<D>::NT : Tab<D>::NE;
    static_assert(NFAC <= 16 && Tab<D>::NE <= 16, "field queue too small");
    constexpr uint32_t GRP[3] = {1u, ((1u << NFAC) - 1u) << 1, D == 3 ? ((1u << Tab<D>::NE) - 1u) << (1 + NFAC) : 0u};
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *mq = aq[wib];
    uint16_t *cw = fq[wib];
    const unsigned long long nw = (c.G.n + 31ull) / 32;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    for (unsigned long long w0 = warp * 32; w0 < nw; w0 += nwarps * 32) {
        uint32_t mine = w0 + lane < nw ? c.Mbits[w0 + lane] : 0u;
        const unsigned cnt = __popc(mine);
        unsigned pre = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= (unsigned)o) pre += y;
        }
        const unsigned total = __shfl_sync(0xffffffffu, pre, 31);
        if (total == 0) continue;
        unsigned at = pre - cnt;
        const uint32_t base = (uint32_t)((w0 + lane) * 32);
        while (mine) {
            const int k = __ffs(mine) - 1;
            mine &= mine - 1;
            mq[at++] = base + (uint32_t)k;
        }
        __syncwarp();
        for (unsigned k0 = 0; k0 < total; k0 += 32) {
            uint32_t m0 = 0;
            if (k0 + lane < total) {
                const uint32_t p = mq[k0 + lane];
                m0 = node_target_mask<D>(__ldg(c.code_f + p), c.code_g[p]);
            }
#pragma unroll
            for (int gi = 0; gi < 3; gi++) {
                uint32_t m = m0 & GRP[gi];
                if (!__any_sync(0xffffffffu, m != 0)) continue;
                const unsigned nc = __popc(m);
                unsigned cpre = nc;
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, cpre, o);
                    if (lane >= (unsigned)o) cpre += y;
                }
                const unsigned ctot = __shfl_sync(0xffffffffu, cpre, 31);
                unsigned ca = cpre - nc;
                while (m) {
                    const int k = __ffs(m) - 1;
                    m &= m - 1;
                    cw[ca++] = (uint16_t)((lane << 5) | (unsigned)k);
                }
                __syncwarp();
                for (unsigned j = lane; j < ctot; j += 32) {
                    const unsigned e = cw[j];
                    const uint32_t p = mq[k0 + (e >> 5)];
                    node_target_item<D>(cc, p, __ldg(c.code_f + p), (int)(e & 31u));
                }
                __syncwarp();
            }
        }
        __syncwarp();
    }
    tally_end(tally, c);
}

// the separatrix dirty set as a list (its bits are set by the refreshes since the last S-pass)
__global__ void k_sd_list(Ctx c, unsigned long long *nSD)
{
    for_each_set(c.sDbits, c.G.n, [&](uint32_t p) { c.sDlist[list_slot(nSD)] = p; });
}

__global__ void k_sd_clear(Ctx c, unsigned long long *nSD)
{
    const unsigned long long n = *nSD;
    GRID_STRIDE(i, n) c.sDbits[c.sDlist[i] >> 5] = 0;
}

// count pass (out == nullptr): one atomic per block; fill pass: staged appends
// separatrix seeds of f, all kinds in one pass over the codes: kind 0 = 1-saddle endpoint
// vertices (descending), 1 = top cofacets of (D-1)-saddles (ascending), 2 = 2-saddle
// triangles (3D).  With out == nullptr only count[kind] is accumulated.
struct SeedOut {
    uint32_t *out[3];
    unsigned long long cap[3];   // entries each list holds; a seed past the end is not written
};

template <int D>
__global__ void k_seeds(const uint64_t *code, Grid G, SeedOut so, unsigned long long *count)
{
    constexpr int NK = D == 3 ? 3 : 2;
    if (!so.out[0]) {
        unsigned long long local[3] = {0, 0, 0};
        GRID_STRIDE(p, G.n)
        for (int k = 0; k < NK; k++) seeds_anchor<D>(code, G, (uint32_t)p, k, [&](uint32_t) { local[k]++; });
        __shared__ unsigned long long warp_sum[3][TPB / 32];
        for (int k = 0; k < NK; k++) {
            unsigned long long v = local[k];
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) warp_sum[k][threadIdx.x >> 5] = v;
        }
        __syncthreads();
        if (threadIdx.x < NK) {
            unsigned long long t = 0;
            for (int w = 0; w < TPB / 32; w++) t += warp_sum[threadIdx.x][w];
            if (t) atomicAdd(count + threadIdx.x, t);
        }
        return;
    }
    // Every thread counts its anchor's seeds by kind; a block scan gives each thread its
    // offsets and one atomic per block and kind reserves the block's range; then the thread
    // derives its seeds again from the code and writes them there.  (Seeds are not rare: ~3
    // per anchor in a noisy field, and one shared atomic per seed queued up.)
    __shared__ unsigned wsum[NK][TPB / 32];
    __shared__ unsigned long long base[NK];
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    BLOCK_ROUNDS(b, G.n)
    {
        const unsigned long long p = b + threadIdx.x;
        unsigned cnt[NK], off[NK];
        for (int k = 0; k < NK; k++) {
            cnt[k] = 0;
            if (p < G.n) seeds_anchor<D>(code, G, (uint32_t)p, k, [&](uint32_t) { cnt[k]++; });
            unsigned incl = cnt[k];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (unsigned)o) incl += y;
            }
            off[k] = incl - cnt[k];
            if (lane == 31) wsum[k][wib] = incl;
        }
        __syncthreads();
        if (threadIdx.x < NK) {
            unsigned long long t = 0;
            for (int w = 0; w < TPB / 32; w++) {
                const unsigned x = wsum[threadIdx.x][w];
                wsum[threadIdx.x][w] = (unsigned)t;       // exclusive prefix of the warps
                t += x;
            }
            base[threadIdx.x] = t ? atomicAdd(count + threadIdx.x, t) : 0;
        }
        __syncthreads();
        if (p < G.n)
            for (int k = 0; k < NK; k++) {
                unsigned long long at = base[k] + wsum[k][wib] + off[k];
                seeds_anchor<D>(code, G, (uint32_t)p, k, [&](uint32_t v) {
                    if (at < so.cap[k]) so.out[k][at] = v;
                    at++;
                });
            }
        __syncthreads();
    }
}

template <int D>
__global__ void k_decode_pairs(const uint64_t *code, Grid G, int64_t *rows, unsigned long long *count, unsigned long long cap)
{
    GRID_STRIDE(p, G.n) decode_pairs<D>(code, G, (uint32_t)p, rows, count, cap);
}

template <int D>
__global__ void k_decode_crit(const uint64_t *code, const uint64_t *ref, Grid G, int64_t *rows, int32_t *dims,
                              unsigned long long *count, unsigned long long cap, Counters *cnt)
{
    GRID_STRIDE(p, G.n) decode_critical<D>(code, ref, G, (uint32_t)p, rows, dims, count, cap, cnt);
}

// per-seed separatrix checks for verification (no sharing between seeds, so the counts
// are per separatrix): rep[8]/rep[9] = separatrices with a pair missing from g's gradient,
// rep[11]/rep[12] = separatrices whose end differs
template <int D> __global__ void k_verify_desc(Ctx c, const uint32_t *seeds, uint32_t n)
{
    const Tab<D> &T = rt_tab<D>();
    GRID_STRIDE(i, n)
    {
        uint32_t u = seeds[i];
        int x, y, z;
        coords(c.G, u, x, y, z);
        bool bad = false;
        for (uint32_t s = 0; s <= c.G.n; s++) {
            const int ff = vfield<D>(__ldg(c.code_f + u));
            if (ff == 15) break;
            if (vfield<D>(c.code_g[u]) != ff) bad = true;
            x += T.nb[ff][0]; y += T.nb[ff][1]; z += T.nb[ff][2];
            u = vid(c.G, x, y, z);
        }
        if (bad) atomicAdd(&c.cnt->rep[8], 1ull);
        if (desc_end<D>(c.code_f, c.G, seeds[i]) != desc_end<D>(c.code_g, c.G, seeds[i])) atomicAdd(&c.cnt->rep[11], 1ull);
    }
}

template <int D> __global__ void k_verify_asc(Ctx c, const uint32_t *seeds, uint32_t n)
{
    GRID_STRIDE(i, n)
    {
        const uint32_t beta = seeds[i];
        int x, y, z, t = (int)(beta % Tab<D>::NTOP);
        coords(c.G, beta / Tab<D>::NTOP, x, y, z);
        const int x0 = x, y0 = y, z0 = z, t0 = t;
        bool bad = false;
        for (uint32_t s = 0; s <= c.G.n * (uint32_t)Tab<D>::NTOP; s++) {
            int fx, fy, fz, ft, ib, jl;
            if (!asc_facet<D>(c.G, c.f, x, y, z, t, c.code_f, fx, fy, fz, ft, ib, jl)) break;
            if (facet_field<D>(c.code_g[vid(c.G, fx, fy, fz)], ft) != 2 + ib) bad = true;
            if (!asc_next<D>(c.G, fx, fy, fz, ft, ib, x, y, z, t)) break;
        }
        if (bad) atomicAdd(&c.cnt->rep[9], 1ull);
        if (asc_end<D>(c.G, c.f, c.code_f, x0, y0, z0, t0) != asc_end<D>(c.G, c.g, c.code_g, x0, y0, z0, t0))
            atomicAdd(&c.cnt->rep[12], 1ull);
    }
}

__global__ void k_max_abs_err(const float *f, const float *g, uint32_t n, unsigned long long *out)
{
    double m = 0.0;
    GRID_STRIDE(i, n) m = fmax(m, fabs((double)g[i] - (double)f[i]));
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// stored form of the edits (Sec. 4.7): q for quantised vertices whose base value needed no
// re-clamping, MSC_QMAP_LOSSLESS otherwise; per-block counts of lossless vertices
__global__ void k_qmap(const float *f, const float *fh, const uint8_t *state, uint32_t n, float xi, int qmax,
                       uint8_t *qmap, uint32_t *block_counts, unsigned long long *nquant)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    int lossless = 0, quant = 0;
    if (i < n) {
        const uint8_t st = state[i];
        const float fc = clamp_base(f[i], fh[i], xi);
        lossless = st > qmax || __float_as_uint(fc) != __float_as_uint(fh[i]);   // qmax 0: every edited vertex
        quant = !lossless && st > 0;
        qmap[i] = lossless ? (uint8_t)MSC_QMAP_LOSSLESS : st;
    }
    const int c = __syncthreads_count(lossless);
    const int q = __syncthreads_count(quant);
    if (threadIdx.x == 0) {
        block_counts[blockIdx.x] = (uint32_t)c;
        if (q) atomicAdd(nquant, (unsigned long long)q);
    }
}

// exclusive scan of the per-block counts (one block)
__global__ void k_scan_blocks(uint32_t *counts, uint32_t nb, unsigned long long *total)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? counts[i] : 0;
        uint32_t x = v;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint32_t s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const uint32_t before = (wid ? warp_sums[wid - 1] : 0) + x - v;
        if (i < nb) counts[i] = carry + before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// write the lossless vertices in ascending order
__global__ void k_lossless_write(const uint8_t *qmap, const float *g, uint32_t n, const uint32_t *offsets,
                                 uint64_t *idx, float *val)
{
    __shared__ uint32_t warp_sums[32];
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const int flag = i < n && qmap[i] == MSC_QMAP_LOSSLESS;
    const unsigned ballot = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sums[wid] = __popc(ballot);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { const uint32_t t = warp_sums[w]; warp_sums[w] = s; s += t; }
    }
    __syncthreads();
    if (flag) {
        const uint32_t pos = offsets[blockIdx.x] + warp_sums[wid] + __popc(ballot & ((1u << lane) - 1u));
        idx[pos] = i;
        if (val) val[pos] = g[i];
    }
}

// ---- packed edit record (Sec. 4.7): b bits per vertex in groups of 8 vertices (b bytes),
// vertex 8k+j of group k in bits [j*b, j*b+b) of the group's little-endian integer; a
// lossless vertex is the escape code 2^b - 1
__global__ void k_pack_q(const uint8_t *qmap, uint64_t n, int b, uint8_t *bits)
{
    const uint64_t groups = (n + 7) / 8;
    const uint32_t esc = (1u << b) - 1u;
    GRID_STRIDE(k, groups)
    {
        uint32_t acc = 0;
        for (int j = 0; j < 8; j++) {
            const uint64_t v = 8 * k + j;
            if (v >= n) break;
            const uint32_t q = qmap[v];
            acc |= (q == MSC_QMAP_LOSSLESS ? esc : q) << (j * b);
        }
        for (int i = 0; i < b; i++) bits[k * b + i] = (uint8_t)(acc >> (8 * i));
    }
}

__global__ void k_unpack_q(const uint8_t *bits, uint64_t n, int b, int qmax, uint8_t *qmap, unsigned long long *bad)
{
    const uint64_t groups = (n + 7) / 8;
    const uint32_t esc = (1u << b) - 1u;
    GRID_STRIDE(k, groups)
    {
        uint32_t acc = 0;
        for (int i = 0; i < b; i++) acc |= (uint32_t)bits[k * b + i] << (8 * i);
        for (int j = 0; j < 8; j++) {
            const uint64_t v = 8 * k + j;
            if (v >= n) break;
            const uint32_t code = (acc >> (j * b)) & esc;
            if (code != esc && (int)code > qmax) atomicAdd(bad, 1ull);
            qmap[v] = code == esc ? (uint8_t)MSC_QMAP_LOSSLESS : (uint8_t)code;
        }
    }
}

// per-block (1024 threads) counts of lossless entries of a q-map, and the quantised total
__global__ void k_qcount(const uint8_t *qmap, uint64_t n, int qmax, uint32_t *block_counts,
                         unsigned long long *nquant, unsigned long long *bad)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const uint8_t q = i < n ? qmap[i] : 0;
    const int lossless = i < n && q == MSC_QMAP_LOSSLESS;
    if (i < n && !lossless && q > qmax) atomicAdd(bad, 1ull);
    const int c = __syncthreads_count(lossless);
    const int nq = __syncthreads_count(i < n && !lossless && q > 0);
    if (threadIdx.x == 0) {
        block_counts[blockIdx.x] = (uint32_t)c;
        if (nq) atomicAdd(nquant, (unsigned long long)nq);
    }
}

// positions where two index lists differ
__global__ void k_count_diff(const uint64_t *a, const uint64_t *b, uint64_t n, unsigned long long *bad)
{
    unsigned long long local = 0;
    GRID_STRIDE(i, n) local += a[i] != b[i];
    if (local) atomicAdd(bad, local);
}

// decompression side: g = f_hat - fl(q * step) (one rounding each), lossless values scattered
__global__ void k_apply_q(const float *fh, const uint8_t *qmap, uint32_t n, float step, float *g)
{
    GRID_STRIDE(i, n)
    {
        const uint8_t q = qmap[i];
        g[i] = q == MSC_QMAP_LOSSLESS ? fh[i] : __fsub_rn(fh[i], __fmul_rn((float)q, step));
    }
}

__global__ void k_apply_lossless(const uint64_t *idx, const float *val, uint64_t n, float *g)
{
    GRID_STRIDE(i, n) g[idx[i]] = val[i];
}

// ------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------
// Device buffers come from the stream-ordered allocator (the device's default memory pool),
// ordered on the stream of the entry point that is running on this thread.  Unlike
// cudaMalloc/cudaFree, allocating or freeing then never waits for work that other jobs
// have queued on other streams.  Every entry point synchronizes its stream before it
// returns, so a buffer allocated in one call is ready for any stream in a later call.
thread_local cudaStream_t g_alloc_stream = nullptr;
thread_local const std::atomic<int> *g_cancel = nullptr;   // set by a serving slot for its job

struct AllocOn {
    cudaStream_t prev;
    explicit AllocOn(cudaStream_t s) : prev(g_alloc_stream) { g_alloc_stream = s; }
    ~AllocOn() { g_alloc_stream = prev; }
};

// The stream of an entry point: orders its allocations, and is synchronized when the entry
// point returns, on success and on every error path alike.  Declared before the entry
// point's buffers, so that their stream-ordered frees are queued before that final wait.
struct EntryStream {
    AllocOn on;
    cudaStream_t s;
    explicit EntryStream(cudaStream_t st) : on(st), s(st) {}
    ~EntryStream()
    {
        cudaStreamSynchronize(s);
        cudaGetLastError();
    }
};

// Page-locked host buffers for the edit records the library hands out.  A device-to-host
// copy into pageable memory runs several times slower than into page-locked memory, and
// pinning fresh memory is slow too, so the buffers msc_free_edits gives back are kept for
// the next record (up to PINNED_IDLE_MAX bytes; msc_release_cached_memory frees them).
constexpr size_t PINNED_IDLE_MAX = 8ull << 30;
struct PinnedCache {
    std::mutex mu;
    std::unordered_map<void *, size_t> live;   // handed out, with their capacity
    std::multimap<size_t, void *> idle;        // given back, by capacity
    size_t idle_bytes = 0;
};
PinnedCache &pinned_cache()
{
    static PinnedCache pc;
    return pc;
}

// a host buffer of at least `bytes` (page-locked when possible); nullptr if none
void *host_take(size_t bytes)
{
    bytes = std::max<size_t>(bytes, 64);
    PinnedCache &pc = pinned_cache();
    {
        std::lock_guard<std::mutex> lk(pc.mu);
        auto it = pc.idle.lower_bound(bytes);
        if (it != pc.idle.end() && it->first <= 2 * bytes + (1u << 20)) {
            void *p = it->second;
            pc.live[p] = it->first;
            pc.idle_bytes -= it->first;
            pc.idle.erase(it);
            return p;
        }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return malloc(bytes);   // not in the cache: freed with free()
    }
    std::lock_guard<std::mutex> lk(pc.mu);
    pc.live[p] = bytes;
    return p;
}

void host_give(void *p)
{
    if (!p) return;
    PinnedCache &pc = pinned_cache();
    std::lock_guard<std::mutex> lk(pc.mu);
    auto it = pc.live.find(p);
    if (it == pc.live.end()) {
        free(p);
        return;
    }
    const size_t cap = it->second;
    pc.live.erase(it);
    if (pc.idle_bytes + cap > PINNED_IDLE_MAX) {
        cudaFreeHost(p);
        return;
    }
    pc.idle.emplace(cap, p);
    pc.idle_bytes += cap;
}

void host_trim()
{
    PinnedCache &pc = pinned_cache();
    std::lock_guard<std::mutex> lk(pc.mu);
    for (auto &kv : pc.idle) cudaFreeHost(kv.second);
    pc.idle.clear();
    pc.idle_bytes = 0;
}

// ------------------------------------------------------------------------------------
// copies between pageable host memory and the device
// ------------------------------------------------------------------------------------
// A cudaMemcpy from or to pageable host memory runs at a few GB/s.  The library instead moves
// such data through page-locked staging chunks: host threads copy one chunk between the
// caller's memory and a staging buffer while the copy engine moves another between the
// staging buffer and the device.

// A fixed pool of host threads that copy disjoint parts of one buffer.
class HostCopyPool {
  public:
    static HostCopyPool &get()
    {
        static HostCopyPool pool;
        return pool;
    }
    // dst[0, n) = src[0, n), split over the pool's threads and the caller
    void copy(void *dst, const void *src, size_t n)
    {
        constexpr size_t PART = 1u << 20;
        const size_t parts = (n + PART - 1) / PART;
        if (workers_.empty() || parts < 2) {
            memcpy(dst, src, n);
            return;
        }
        std::lock_guard<std::mutex> one(job_mu_);     // one job at a time
        {
            std::lock_guard<std::mutex> lk(mu_);
            dst_ = (char *)dst;
            src_ = (const char *)src;
            n_ = n;
            part_ = PART;
            parts_ = parts;
            next_.store(0);
            left_.store(parts);
            gen_++;
        }
        cv_.notify_all();
        run_parts();
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return left_.load() == 0; });
    }
    ~HostCopyPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : workers_) t.join();
    }

  private:
    HostCopyPool()
    {
        // every core but the caller's, up to 15: one thread moves ~14 GB/s on a Grace host, and
        // the copy engine takes ~200 GB/s from page-locked memory
        const unsigned hc = std::thread::hardware_concurrency();
        const unsigned n = hc > 2 ? std::min(15u, hc - 1) : 0;
        for (unsigned i = 0; i < n; i++) workers_.emplace_back([this] { loop(); });
    }
    void run_parts()
    {
        for (;;) {
            const size_t i = next_.fetch_add(1);
            if (i >= parts_) return;
            const size_t off = i * part_, len = std::min(part_, n_ - off);
            memcpy(dst_ + off, src_ + off, len);
            if (left_.fetch_sub(1) == 1) {
                std::lock_guard<std::mutex> lk(mu_);
                done_cv_.notify_all();
            }
        }
    }
    void loop()
    {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
            }
            run_parts();
        }
    }
    std::vector<std::thread> workers_;
    std::mutex job_mu_, mu_;
    std::condition_variable cv_, done_cv_;
    char *dst_ = nullptr;
    const char *src_ = nullptr;
    size_t n_ = 0, part_ = 1, parts_ = 0;
    std::atomic<size_t> next_{0}, left_{0};
    uint64_t gen_ = 0;
    bool stop_ = false;
};

enum class MemKind { Device, PinnedHost, PageableHost };

MemKind mem_kind(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return MemKind::PageableHost;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return MemKind::Device;
    if (a.type == cudaMemoryTypeHost) return MemKind::PinnedHost;
    return MemKind::PageableHost;
}

constexpr size_t STAGE_CHUNK = 32u << 20;   // bytes per staging chunk
constexpr int STAGE_BUFS = 3;               // chunks in flight

struct Staging {
    void *buf[STAGE_BUFS] = {};
    cudaEvent_t ev[STAGE_BUFS] = {};
    bool pinned_ok = true;
    ~Staging()
    {
        for (int i = 0; i < STAGE_BUFS; i++) {
            if (ev[i]) { cudaEventSynchronize(ev[i]); cudaEventDestroy(ev[i]); }
            host_give(buf[i]);
        }
        cudaGetLastError();
    }
    cudaError_t init(size_t chunk)
    {
        for (int i = 0; i < STAGE_BUFS; i++) {
            buf[i] = host_take(chunk);
            if (!buf[i]) return cudaErrorMemoryAllocation;
            cudaError_t e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

// n bytes from src (host or device) to device memory dst, ordered on stream s.  From pageable
// host memory the call returns once src may be reused (every chunk has been staged).
cudaError_t copy_to_device(void *dst, const void *src, size_t n, cudaStream_t s)
{
    const MemKind k = mem_kind(src);
    if (k == MemKind::Device) return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, s);
    // (no direct path from pageable memory, even where the device reads host page tables: its
    // rate depends on how the host backs the pages, 190 GB/s on a fresh process, e2e at 512^3
    // 1.3 GB/s direct against 2.4 GB/s staged after other work had run on the host)
    if (k == MemKind::PinnedHost || n <= STAGE_CHUNK) return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
    Staging st;
    cudaError_t e = st.init(STAGE_CHUNK);
    if (e != cudaSuccess) return e;
    HostCopyPool &pool = HostCopyPool::get();
    for (size_t off = 0, i = 0; off < n; off += STAGE_CHUNK, i++) {
        const int b = (int)(i % STAGE_BUFS);
        const size_t len = std::min(STAGE_CHUNK, n - off);
        if ((e = cudaEventSynchronize(st.ev[b])) != cudaSuccess) return e;    // its last copy is done
        pool.copy(st.buf[b], (const char *)src + off, len);
        if ((e = cudaMemcpyAsync((char *)dst + off, st.buf[b], len, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(st.ev[b], s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// n bytes from device memory src to dst (host or device), ordered on stream s.  To pageable
// host memory the call waits for the copy and returns when dst holds the data.
cudaError_t copy_from_device(void *dst, const void *src, size_t n, cudaStream_t s)
{
    const MemKind k = mem_kind(dst);
    if (k == MemKind::Device) return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, s);
    // (no direct path here either: the device's first writes to a host buffer run slowly while
    // it maps the pages, 27 GB/s for a fresh 512 MB array)
    if (k == MemKind::PinnedHost || n <= STAGE_CHUNK) return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s);
    Staging st;
    cudaError_t e = st.init(STAGE_CHUNK);
    if (e != cudaSuccess) return e;
    HostCopyPool &pool = HostCopyPool::get();
    const size_t nchunk = (n + STAGE_CHUNK - 1) / STAGE_CHUNK;
    auto drain = [&](size_t j) -> cudaError_t {    // chunk j has been queued: move it out
        const int b = (int)(j % STAGE_BUFS);
        cudaError_t r = cudaEventSynchronize(st.ev[b]);
        if (r != cudaSuccess) return r;
        pool.copy((char *)dst + j * STAGE_CHUNK, st.buf[b], std::min(STAGE_CHUNK, n - j * STAGE_CHUNK));
        return cudaSuccess;
    };
    for (size_t i = 0; i < nchunk; i++) {
        const int b = (int)(i % STAGE_BUFS);
        if (i >= (size_t)STAGE_BUFS && (e = drain(i - STAGE_BUFS)) != cudaSuccess) return e;
        const size_t off = i * STAGE_CHUNK, len = std::min(STAGE_CHUNK, n - off);
        if ((e = cudaMemcpyAsync(st.buf[b], (const char *)src + off, len, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(st.ev[b], s)) != cudaSuccess) return e;
    }
    for (size_t j = nchunk > (size_t)STAGE_BUFS ? nchunk - STAGE_BUFS : 0; j < nchunk; j++)
        if ((e = drain(j)) != cudaSuccess) return e;
    return cudaSuccess;
}

// The library's own stream-ordered memory pool on each device.  Device memory that a handle
// frees stays in the pool (release threshold: unlimited) for the next handle, so a sequence
// of prepare / fix / destroy calls does not map and unmap its working set every time;
// msc_release_cached_memory hands it back to the driver.
std::mutex g_pool_mu;
std::vector<std::pair<int, cudaMemPool_t>> g_pools;

cudaMemPool_t lib_pool()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto &dp : g_pools)
        if (dp.first == dev) return dp.second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) { cudaGetLastError(); pool = nullptr; }
    if (pool) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pools.emplace_back(dev, pool);
    return pool;
}

// (triangle, delta) pairs a saddle-saddle spill queue holds: one per vertex, at least 1 M (a
// small field whose walks spill often, for instance under lowered walk limits, still fits)
uint64_t ovf_pairs(uint64_t n) { return std::max<uint64_t>(n + 1, 1ull << 20); }

// walk limits (msc_set_walk_limits): the saddle-saddle stack entries a warp uses, the steps
// a thread walks before spilling
std::atomic<uint32_t> g_walk_stack{(uint32_t)SS_WARP_STACK}, g_walk_steps{TRI_LOCAL_STEPS};

// allocation-failure injection (msc_inject_alloc_failures): the count of allocations still
// allowed before failures start, and the failures left to inject
std::atomic<uint64_t> g_inject_after{0}, g_inject_left{0}, g_injected{0};

bool inject_alloc_failure()
{
    if (g_inject_left.load(std::memory_order_relaxed) == 0) return false;
    uint64_t a = g_inject_after.load();
    while (a > 0)
        if (g_inject_after.compare_exchange_weak(a, a - 1)) return false;
    uint64_t l = g_inject_left.load();
    while (l > 0)
        if (g_inject_left.compare_exchange_weak(l, l - 1)) {
            g_injected.fetch_add(1);
            return true;
        }
    return false;
}

template <class T> struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    cudaError_t alloc(size_t count)
    {
        if (count <= n && p) return cudaSuccess;
        release();
        if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
        cudaMemPool_t pool = lib_pool();
        const size_t bytes = (count ? count : 1) * sizeof(T);
        cudaError_t e = pool ? cudaMallocFromPoolAsync((void **)&p, bytes, pool, g_alloc_stream)
                             : cudaMallocAsync((void **)&p, bytes, g_alloc_stream);
        if (e == cudaSuccess) n = count;
        else p = nullptr;
        return e;
    }
    void release()
    {
        if (p) cudaFreeAsync(p, g_alloc_stream);
        p = nullptr;
        n = 0;
    }
};

}  // namespace
struct msc_handle;
namespace {
void kbeg(msc_handle *h, int cls, cudaStream_t s);
void kend(msc_handle *h, cudaStream_t s);
#define KL(h, cls, s, ...)   \
    do {                     \
        kbeg(h, cls, s);     \
        __VA_ARGS__;         \
        kend(h, s);          \
    } while (0)

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

msc_status check_dims(int nx, int ny, int nz)
{
    if (nx < 2 || ny < 2 || nz < 1) return fail(MSC_ERR_INVALID_ARG, "dims must satisfy nx, ny >= 2 and nz >= 1 (got %d %d %d)", nx, ny, nz);
    const unsigned long long n = (unsigned long long)nx * ny * nz;
    if (n >= (1ull << 31)) return fail(MSC_ERR_INVALID_ARG, "grid too large: %llu vertices (limit 2^31)", n);
    // per-anchor cell ids (anchor * 12 + type) must fit in 32 bits
    if (nz > 1 && n * 12ull >= (1ull << 32)) return fail(MSC_ERR_INVALID_ARG, "3D grid too large for 32-bit cell ids");
    return MSC_OK;
}

msc_status device_ready()
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(MSC_ERR_NO_DEVICE, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    return MSC_OK;
}

// copy (host or device) input to a device buffer and check all values are finite
msc_status upload_field(msc_handle *h, const float *src, size_t n, float *dst, unsigned long long *bad_dev, cudaStream_t s,
                        const char *what)
{
    if (!src) return fail(MSC_ERR_INVALID_ARG, "%s is NULL", what);
    CK(copy_to_device(dst, src, n * sizeof(float), s));
    CK(cudaMemsetAsync(bad_dev, 0, sizeof(unsigned long long), s));
    KL(h, MSC_K_OTHER, s, k_count_nonfinite<<<grid_occ((const void *)k_count_nonfinite, n), TPB, 0, s>>>(dst, (uint32_t)n, bad_dev));
    CK(cudaGetLastError());
    unsigned long long bad = 0;
    CK(cudaMemcpyAsync(&bad, bad_dev, sizeof bad, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (bad) return fail(MSC_ERR_INVALID_ARG, "%s has %llu non-finite values", what, bad);
    return MSC_OK;
}

void fill_defaults(msc_options *o)
{
    o->tier = 4;
    o->q_max = 6;
    o->max_iters = 100000;
    o->exact_fallback = 1;
    o->tile_x = o->tile_y = o->tile_z = 0;
    o->stream = nullptr;
    o->record_trace = 0;
    o->profile = 0;
    o->small_round = 0;
    o->edit_mode = MSC_EDITS_QUANTIZED;
    o->cluster_round = 0;
}

msc_status check_options(const msc_options *o)
{
    if (o->tier < 1 || o->tier > 4) return fail(MSC_ERR_INVALID_ARG, "tier must be 1..4 (got %d)", o->tier);
    if (o->q_max < 1 || o->q_max > 7) return fail(MSC_ERR_INVALID_ARG, "q_max must be 1..7 (got %d)", o->q_max);
    if (o->max_iters < 0) return fail(MSC_ERR_INVALID_ARG, "max_iters must be >= 0");
    if (o->small_round < 0) return fail(MSC_ERR_INVALID_ARG, "small_round must be >= 0");
    if (o->cluster_round < 0) return fail(MSC_ERR_INVALID_ARG, "cluster_round must be >= 0");
    if (o->edit_mode != MSC_EDITS_QUANTIZED && o->edit_mode != MSC_EDITS_FLOAT)
        return fail(MSC_ERR_INVALID_ARG, "edit_mode must be 0 (quantized) or 1 (float)");
    if (o->edit_mode == MSC_EDITS_FLOAT && o->q_max > 6)
        return fail(MSC_ERR_INVALID_ARG, "floating edits need q_max <= 6 (got %d)", o->q_max);
    return MSC_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------
// the handle
// ------------------------------------------------------------------------------------
struct msc_handle {
    Grid G{};
    int D = 3;
    DevBuf<float> f;
    DevBuf<uint64_t> code_f;
    DevBuf<uint64_t> low_f;   // 3D: lowest vertex slot of every triangle and tetrahedron under f
    DevBuf<uint32_t> seeds_desc, seeds_asc, seeds_ss;
    uint32_t n_desc = 0, n_asc = 0, n_ss = 0;
    // fix state (allocated on first use)
    DevBuf<float> fhat, g, gprev;
    DevBuf<uint8_t> state;
    DevBuf<uint64_t> code_g;
    DevBuf<uint32_t> Tbits, Xbits, Dbits, Tlist, Xlist, Dlist, Elist, Mbits, Cbits, Csum, Cblk, Cblk2;
    DevBuf<GridBarrier> bar;
    int rounds_grid = 0;   // blocks of the persistent round kernel (0: one per SM)
    uint64_t cluster_launches = 0, cluster_rounds = 0;   // the round kernel's cluster form
    DevBuf<unsigned long long> seed_count;   // seeds counted by prepare's dense pass over f
    bool seeds_counted = false;
    int tile_req = -1;     // tile shape of the dense 3D gradient the current call asks for (-1: tuned)
    int tile_used = -1;    // the shape its last dense pass ran with
    DevBuf<uint32_t> vis_v, vis_top, vis_tri, ovf0, ovf1;
    DevBuf<uint32_t> ns_v, ns_top, ns_tri, ns_dead;
    DevBuf<uint32_t> sDbits, sDlist;
    DevBuf<Counters> cnt;
    DevBuf<LoopState> ls;
    DevBuf<int64_t> trace;
    cudaStream_t cap_stream = nullptr;   // graphs are captured on this stream
    DevBuf<unsigned long long> nM;   // scratch counters of uploads
    bool fix_ready = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // launch statistics
    unsigned prof_mask = 0;   // kernel classes timed in the current call
    bool last_timed = false;  // the launch opened by kbeg is being timed
    unsigned long long launches[12] = {};
    unsigned long long timed[12] = {};
    unsigned long long items[12] = {};
    unsigned long long round_work[3] = {};   // edit, refresh, cpass items of the round kernel
    unsigned long long round_phase_ns[4] = {};   // device time per phase of the round kernel
    double ms[12] = {};
    struct Pend {
        cudaEvent_t a, b;
        int cls;
    };
    std::vector<Pend> pend;
    std::vector<cudaEvent_t> pool;
    ~msc_handle()
    {
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (auto &p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

namespace {

cudaEvent_t take_event(msc_handle *h)
{
    if (!h->pool.empty()) { cudaEvent_t e = h->pool.back(); h->pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void kbeg(msc_handle *h, int cls, cudaStream_t s)
{
    if (!h) return;
    h->launches[cls]++;
    h->last_timed = (h->prof_mask >> cls) & 1u;
    if (!h->last_timed) return;
    msc_handle::Pend p{take_event(h), take_event(h), cls};
    cudaEventRecord(p.a, s);
    h->pend.push_back(p);
}

void kend(msc_handle *h, cudaStream_t s)
{
    if (!h || !h->last_timed || h->pend.empty()) return;
    cudaEventRecord(h->pend.back().b, s);
    h->last_timed = false;
}

// resolve the timed launches of a finished call
void prof_flush(msc_handle *h)
{
    for (auto &p : h->pend) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            h->ms[p.cls] += ms;
            h->timed[p.cls]++;
        }
        h->pool.push_back(p.a);
        h->pool.push_back(p.b);
    }
    h->pend.clear();
    cudaGetLastError();
}

size_t words(size_t bits) { return (bits + 31) / 32; }

msc_status alloc_fix_state(msc_handle *h)
{
    if (h->fix_ready) return MSC_OK;
    const size_t n = h->G.n;
    const int ntop = h->D == 3 ? 6 : 2;
    CK(h->fhat.alloc(n));
    CK(h->g.alloc(n));
    CK(h->state.alloc(n));
    CK(h->code_g.alloc(n));
    CK(h->Tbits.alloc(words(n)));
    CK(h->Xbits.alloc(words(n)));
    CK(h->Dbits.alloc(words(n)));
    CK(h->Tlist.alloc(n));
    CK(h->Xlist.alloc(n));
    CK(h->Dlist.alloc(n));
    CK(h->Elist.alloc(n));
    CK(h->gprev.alloc(n));
    CK(h->Mbits.alloc(words(n)));
    CK(h->Cbits.alloc(words(n)));
    CK(h->Csum.alloc(csum_words((uint32_t)n)));
    CK(h->Cblk.alloc(csum_words((uint32_t)n) * 32));
    CK(h->Cblk2.alloc(csum_words((uint32_t)n) * 32));
    CK(h->bar.alloc(1));
    CK(cudaMemsetAsync(h->bar.p, 0, sizeof(GridBarrier), g_alloc_stream));
    CK(h->vis_v.alloc(words(n)));
    CK(h->vis_top.alloc(words(n * ntop)));
    if (h->D == 3) {
        CK(h->vis_tri.alloc(words(n * 12)));
        CK(h->ovf0.alloc(2 * ovf_pairs(n)));
        CK(h->ovf1.alloc(2 * ovf_pairs(n)));
    }
    CK(h->ns_v.alloc(node_words(n + 4)));
    CK(h->ns_top.alloc(node_words(n * ntop + 4)));
    if (h->D == 3) {
        CK(h->ns_tri.alloc(node_words(n * 12 + 4)));
        CK(h->ns_dead.alloc(node_words(n * 7 + 4)));
    }
    CK(h->sDbits.alloc(words(n)));
    CK(h->sDlist.alloc(n));
    CK(cudaMemsetAsync(h->sDbits.p, 0, h->sDbits.n * 4, g_alloc_stream));
    CK(h->cnt.alloc(2));   // [0]: the round graphs and the S-pass; [0], [1]: persistent rounds
    CK(h->nM.alloc(8));
    CK(h->ls.alloc(1));
    CK(cudaMemsetAsync(h->Tbits.p, 0, h->Tbits.n * 4, g_alloc_stream));
    CK(cudaMemsetAsync(h->Xbits.p, 0, h->Xbits.n * 4, g_alloc_stream));
    CK(cudaMemsetAsync(h->Dbits.p, 0, h->Dbits.n * 4, g_alloc_stream));
    h->fix_ready = true;
    return MSC_OK;
}

// steps a vertex may take before the floor: q_max (Eq. 2), or, for floating edits, more than
// the 2^(q_max+1) steps of xi / 2^q_max that fit between f + xi and f - xi (no cap)
constexpr int FLOAT_EDIT_CAP = 0xEF;

Ctx make_ctx(msc_handle *h, int tier, int qmax, int exact_fallback, float xi, int edit_mode = MSC_EDITS_QUANTIZED)
{
    Ctx c{};
    c.G = h->G;
    c.tier = tier;
    c.qmax = qmax;
    c.qcap = edit_mode == MSC_EDITS_FLOAT ? FLOAT_EDIT_CAP : qmax;
    c.exact_fallback = exact_fallback;
    c.xi = xi;
    c.step = xi / (float)(1 << qmax);
    c.f = h->f.p;
    c.fhat = h->fhat.p;
    c.g = h->g.p;
    c.state = h->state.p;
    c.code_f = h->code_f.p;
    c.low_f = h->low_f.p;
    c.code_g = h->code_g.p;
    c.Tbits = h->Tbits.p; c.Xbits = h->Xbits.p; c.Dbits = h->Dbits.p;
    c.Tlist = h->Tlist.p; c.Xlist = h->Xlist.p; c.Dlist = h->Dlist.p;
    c.Elist = h->Elist.p;
    c.gprev = h->gprev.p;
    c.vis_v = h->vis_v.p; c.vis_top = h->vis_top.p; c.vis_tri = h->vis_tri.p;
    c.ovf_cap = (uint32_t)ovf_pairs(h->G.n);
    c.ss_stack_cap = g_walk_stack.load();
    c.tri_local_steps = g_walk_steps.load();
    c.cnt = h->cnt.p;
    c.ns_v = h->ns_v.p; c.ns_top = h->ns_top.p; c.ns_tri = h->ns_tri.p; c.ns_dead = h->ns_dead.p;
    c.sDbits = h->sDbits.p; c.sDlist = h->sDlist.p;
    c.ls = h->ls.p;
    c.Mbits = h->Mbits.p;
    c.Cbits = h->Cbits.p;
    c.Csum = h->Csum.p;
    c.Cblk = h->Cblk.p;
    c.trace = nullptr;
    c.tally = nullptr;
    return c;
}

// ------------------------------------------------------------------------------------
// tile shapes of k_eval_tile and their autotuner
// ------------------------------------------------------------------------------------
// The shapes instantiated: 32 x TY anchors per block, ZS planes per z-slab.  Deeper slabs
// recompute fewer halo planes (3 per slab) but give fewer blocks; taller tiles share more of
// their halo rows but hold more shared memory per block.  The first dense pass of a 3D grid
// shape on a device times every shape once on its input (all shapes write the same codes) and
// keeps the fastest for that (device, nx, ny, nz); msc_options.tile_* picks one instead.
using TileFn = void (*)(const float *, Grid, uint64_t *, const uint64_t *, uint32_t *, uint32_t *, uint32_t *, int,
                        uint64_t *, unsigned long long *);
struct TileShape {
    int ty, zs, nt;
    TileFn fn;
};
const TileShape TILE_SHAPES[] = {
    {8, 16, 256, k_eval_tile<8, 16, 3>},
    {8, 8, 256, k_eval_tile<8, 8, 3>},
    {8, 32, 256, k_eval_tile<8, 32, 3>},
    {4, 16, 128, k_eval_tile<4, 16, 6>},
    {16, 16, 512, k_eval_tile<16, 16, 1>},
};
constexpr int N_TILE_SHAPES = (int)(sizeof(TILE_SHAPES) / sizeof(TILE_SHAPES[0]));

struct TileTuning {
    int best = 0;
    float ms[N_TILE_SHAPES] = {};
};
std::mutex g_tile_mu;
std::map<std::tuple<int, int, int, int>, TileTuning> g_tile_tuned;

// the shape index the options ask for: -1 = tuned, else an instantiated shape
msc_status tile_request(const msc_options &o, int *req)
{
    *req = -1;
    if (!o.tile_x && !o.tile_y && !o.tile_z) return MSC_OK;
    for (int i = 0; i < N_TILE_SHAPES; i++)
        if (o.tile_x == 32 && o.tile_y == TILE_SHAPES[i].ty && o.tile_z == TILE_SHAPES[i].zs) {
            *req = i;
            return MSC_OK;
        }
    return fail(MSC_ERR_INVALID_ARG, "tile %dx%dx%d is not instantiated (32 x {4,8,16} x {8,16,32} as listed by "
                "msc_tile_report; 0 = tuned)", o.tile_x, o.tile_y, o.tile_z);
}

void launch_tile(int i, const float *v, Grid G, uint64_t *out, cudaStream_t s, const uint64_t *ref, uint32_t *mbits,
                 uint32_t *cbits, uint32_t *csum, int tier, uint64_t *low, unsigned long long *seeds = nullptr)
{
    const TileShape &t = TILE_SHAPES[i];
    const dim3 grid((G.nx + 31) / 32, (G.ny + t.ty - 1) / t.ty, (G.nz + t.zs - 1) / t.zs);
    t.fn<<<grid, t.nt, 0, s>>>(v, G, out, ref, mbits, cbits, csum, tier, low, seeds);
}

// the dense gradient of a 3D grid with the requested tile shape, or the tuned one (tuning it
// on the first pass of this grid shape on this device)
msc_status eval_tile(msc_handle *h, const float *v, Grid G, uint64_t *out, cudaStream_t s, const uint64_t *ref,
                     uint32_t *mbits, uint32_t *cbits, uint32_t *csum, int tier, uint64_t *low)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int shape = h ? h->tile_req : -1;     // no handle (introspection calls): the tuned shape
    if (shape < 0) {
        const auto key = std::make_tuple(dev, G.nx, G.ny, G.nz);
        {
            std::lock_guard<std::mutex> lk(g_tile_mu);
            auto it = g_tile_tuned.find(key);
            if (it != g_tile_tuned.end()) shape = it->second.best;
        }
        if (shape < 0) {
            // one untimed launch, then every shape once; each writes the same codes to out
            TileTuning tt;
            cudaEvent_t e[N_TILE_SHAPES + 1];
            for (int i = 0; i <= N_TILE_SHAPES; i++) CK(cudaEventCreate(&e[i]));
            launch_tile(0, v, G, out, s, ref, mbits, cbits, csum, tier, low);
            CK(cudaEventRecord(e[0], s));
            for (int i = 0; i < N_TILE_SHAPES; i++) {
                launch_tile(i, v, G, out, s, ref, mbits, cbits, csum, tier, low);
                CK(cudaEventRecord(e[i + 1], s));
            }
            CK(cudaGetLastError());
            CK(cudaEventSynchronize(e[N_TILE_SHAPES]));
            for (int i = 0; i < N_TILE_SHAPES; i++) {
                CK(cudaEventElapsedTime(&tt.ms[i], e[i], e[i + 1]));
                if (tt.ms[i] < tt.ms[tt.best]) tt.best = i;
            }
            for (int i = 0; i <= N_TILE_SHAPES; i++) cudaEventDestroy(e[i]);
            {
                std::lock_guard<std::mutex> lk(g_tile_mu);
                g_tile_tuned.emplace(key, tt);
            }
            if (h) {
                h->launches[MSC_K_DENSE] += N_TILE_SHAPES + 1;
                h->tile_used = tt.best;
            }
            return MSC_OK;
        }
    }
    if (h) h->tile_used = shape;
    // the pass over f in prepare also counts the separatrix seeds (build_seeds then needs
    // only its fill pass); a tuning pass does not, as it runs every shape
    unsigned long long *seeds = h && low && h->seed_count.p ? h->seed_count.p : nullptr;
    if (seeds) {
        CK(cudaMemsetAsync(seeds, 0, 3 * sizeof(unsigned long long), s));
        h->seeds_counted = true;
    }
    KL(h, MSC_K_DENSE, s, launch_tile(shape, v, G, out, s, ref, mbits, cbits, csum, tier, low, seeds));
    CK(cudaGetLastError());
    return MSC_OK;
}

template <int D> msc_status eval_dense(msc_handle *h, const float *v, Grid G, uint64_t *out, cudaStream_t s,
                                       const uint64_t *ref = nullptr, uint32_t *mbits = nullptr,
                                       uint32_t *cbits = nullptr, uint32_t *csum = nullptr, int tier = 4,
                                       uint64_t *low = nullptr)
{
    if constexpr (D == 3) {
        if (ref) {
            CK(cudaMemsetAsync(mbits, 0, ((G.n + 31ull) / 32) * 4, s));
            CK(cudaMemsetAsync(cbits, 0, ((G.n + 31ull) / 32) * 4, s));
        }
        CKS(eval_tile(h, v, G, out, s, ref, mbits, cbits, csum, tier, low));
    } else {
        KL(h, MSC_K_DENSE, s, k_eval_dense<D><<<grid_occ((const void *)k_eval_dense<D>, G.n), TPB, 0, s>>>(v, G, out, ref, mbits, cbits, csum, tier));
    }
    CK(cudaGetLastError());
    return MSC_OK;
}

msc_status eval_dense_any(msc_handle *h, int D, const float *v, Grid G, uint64_t *out, cudaStream_t s, uint64_t *low = nullptr)
{
    return D == 3 ? eval_dense<3>(h, v, G, out, s, nullptr, nullptr, nullptr, nullptr, 4, low) : eval_dense<2>(h, v, G, out, s);
}

template <int D> msc_status build_seeds(msc_handle *h, cudaStream_t s)
{
    DevBuf<unsigned long long> cnt;
    CK(cnt.alloc(3));
    DevBuf<uint32_t> *bufs[3] = {&h->seeds_desc, &h->seeds_asc, &h->seeds_ss};
    uint32_t *ns[3] = {&h->n_desc, &h->n_asc, &h->n_ss};
    unsigned long long n[3] = {0, 0, 0};
    SeedOut so{{nullptr, nullptr, nullptr}, {0, 0, 0}};
    if (h->seeds_counted) {
        CK(cudaMemcpyAsync(n, h->seed_count.p, sizeof n, cudaMemcpyDeviceToHost, s));
    } else {
        CK(cudaMemsetAsync(cnt.p, 0, sizeof n, s));
        KL(h, MSC_K_OTHER, s, k_seeds<D><<<grid_occ((const void *)k_seeds<D>, h->G.n), TPB, 0, s>>>(h->code_f.p, h->G, so, cnt.p));
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(n, cnt.p, sizeof n, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; k++) {
        CK(bufs[k]->alloc(n[k]));
        so.out[k] = bufs[k]->p;
        so.cap[k] = n[k];
        *ns[k] = (uint32_t)n[k];
    }
    CK(cudaMemsetAsync(cnt.p, 0, sizeof n, s));
    KL(h, MSC_K_OTHER, s, k_seeds<D><<<grid_occ((const void *)k_seeds<D>, h->G.n), TPB, 0, s>>>(h->code_f.p, h->G, so, cnt.p));
    CK(cudaGetLastError());
    unsigned long long m[3];
    CK(cudaMemcpyAsync(m, cnt.p, sizeof m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < 3; k++)
        if (m[k] != n[k]) return fail(MSC_ERR_CUDA, "separatrix seed lists: %llu seeds listed, %llu counted", m[k], n[k]);
    cnt.release();
    return MSC_OK;
}

// one S-pass (Sec. 4.4) over the separatrices of f; counters accumulate in h->cnt
template <int D> msc_status s_pass(msc_handle *h, const Ctx &c0, int tier, cudaStream_t s)
{
    Ctx c = c0;
    CK(cudaMemsetAsync(h->vis_v.p, 0, h->vis_v.n * 4, s));
    CK(cudaMemsetAsync(h->vis_top.p, 0, h->vis_top.n * 4, s));
    if (h->n_desc) KL(h, MSC_K_SEP_UPDATE, s, k_desc<D><<<grid_occ((const void *)k_desc<D>, h->n_desc), TPB, 0, s>>>(c, h->seeds_desc.p, h->n_desc));
    if (h->n_asc) KL(h, MSC_K_SEP_UPDATE, s, k_asc<D><<<grid_occ((const void *)k_asc<D>, h->n_asc), TPB, 0, s>>>(c, h->seeds_asc.p, h->n_asc));
    CK(cudaGetLastError());
    if (D == 3 && tier >= 4 && h->n_ss) {
        CK(cudaMemsetAsync(h->vis_tri.p, 0, h->vis_tri.n * 4, s));
        c.ovf_out = h->ovf0.p;
        KL(h, MSC_K_SEP_UPDATE, s, k_ss_seed<<<grid_occ((const void *)k_ss_seed, h->n_ss), TPB, 0, s>>>(c, h->seeds_ss.p, h->n_ss));
        CK(cudaGetLastError());
        uint32_t *in = h->ovf0.p, *out = h->ovf1.p;
        for (int round = 0; round < 1 << 20; round++) {
            Counters hc;
            CK(cudaMemcpyAsync(&hc, h->cnt.p, sizeof hc, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (hc.err) return fail(MSC_ERR_OOM, "saddle-saddle spill queue overflow");
            if (hc.novf == 0) break;
            const unsigned long long zero = 0;
            CK(cudaMemcpyAsync(&h->cnt.p->novf, &zero, sizeof zero, cudaMemcpyHostToDevice, s));
            c.ovf_out = out;
            KL(h, MSC_K_SEP_UPDATE, s, k_ss_spill<<<grid_occ((const void *)k_ss_spill, hc.novf), TPB, 0, s>>>(c, in, (uint32_t)hc.novf));
            CK(cudaGetLastError());
            std::swap(in, out);
        }
    }
    return MSC_OK;
}

// tier-4 S-pass from the persistent separatrix state: built once per fix, then updated at
// the anchors dirtied since the previous S-pass; troublemakers read at the mismatch anchors
template <int D> msc_status s_pass_state(msc_handle *h, Ctx &c, bool &built, unsigned long long *nSD, cudaStream_t s)
{
    c.ovf_out = D == 3 ? h->ovf0.p : nullptr;
    const int spill_cls = built ? MSC_K_SEP_UPDATE : MSC_K_SEP_SEED;
    if (!built) {
        CK(cudaMemsetAsync(h->ns_v.p, NS_FILL, h->ns_v.n * 4, s));
        CK(cudaMemsetAsync(h->ns_top.p, NS_FILL, h->ns_top.n * 4, s));
        if (D == 3) {
            CK(cudaMemsetAsync(h->ns_tri.p, NS_FILL, h->ns_tri.n * 4, s));
            CK(cudaMemsetAsync(h->ns_dead.p, NS_FILL, h->ns_dead.n * 4, s));
        }
        KL(h, MSC_K_SEP_INIT, s, k_node_init<D><<<grid_occ((const void *)k_node_init<D>, h->G.n), TPB, 0, s>>>(c));
        if (h->n_desc) KL(h, MSC_K_SEP_SEED, s, k_node_seed<D><<<grid_occ((const void *)k_node_seed<D>, h->n_desc), TPB, 0, s>>>(c, 0, h->seeds_desc.p, h->n_desc));
        if (h->n_asc) KL(h, MSC_K_SEP_SEED, s, k_node_seed<D><<<grid_occ((const void *)k_node_seed<D>, h->n_asc), TPB, 0, s>>>(c, 1, h->seeds_asc.p, h->n_asc));
        if (D == 3 && h->n_ss) {
            const int ssg = std::min(grid_occ((const void *)k_node_seed_ss, 32ull * h->n_ss), SS_BLOCKS_PER_SM * sm_count());
            KL(h, MSC_K_SEP_SEED, s, k_node_seed_ss<<<ssg, TPB, 0, s>>>(c, h->seeds_ss.p, h->n_ss));
        }
        CK(cudaGetLastError());
        h->items[MSC_K_SEP_INIT] += h->G.n;
        built = true;
        k_set_track<<<1, 1, 0, s>>>(h->ls.p, 1);
    } else {
        CK(cudaMemsetAsync(nSD, 0, sizeof(unsigned long long), s));
        KL(h, MSC_K_SEP_UPDATE, s, k_sd_list<<<grid_occ((const void *)k_sd_list, ((unsigned long long)h->G.n + 31) / 32), TPB, 0, s>>>(c, nSD));
        KL(h, MSC_K_SEP_UPDATE, s, k_node_update<D><<<grid_occ((const void *)k_node_update<D>, h->G.n / 16 + 1), TPB, 0, s>>>(c, nSD));
        CK(cudaGetLastError());
    }
    if (D == 3) {
        uint32_t *in = h->ovf0.p, *out = h->ovf1.p;
        for (int round = 0; round < 1 << 20; round++) {
            Counters hc;
            CK(cudaMemcpyAsync(&hc, h->cnt.p, sizeof hc, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (hc.err) return fail(MSC_ERR_OOM, "separatrix spill queue overflow");
            if (hc.novf == 0) break;
            const unsigned long long zero = 0;
            CK(cudaMemcpyAsync(&h->cnt.p->novf, &zero, sizeof zero, cudaMemcpyHostToDevice, s));
            c.ovf_out = out;
            const int tg = std::min(grid_occ((const void *)k_tri_spill, hc.novf), SS_BLOCKS_PER_SM * sm_count());
            KL(h, spill_cls, s, k_tri_spill<<<tg, TPB, 0, s>>>(c, in, (uint32_t)hc.novf));
            CK(cudaGetLastError());
            std::swap(in, out);
        }
    }
    KL(h, MSC_K_SEP_UPDATE, s, k_sd_clear<<<grid_occ((const void *)k_sd_clear, h->G.n / 16 + 1), TPB, 0, s>>>(c, nSD));
    CK(cudaMemsetAsync(nSD, 0, sizeof(unsigned long long), s));
    KL(h, MSC_K_SEP_TARGETS, s, k_node_targets<D><<<grid_occ((const void *)k_node_targets<D>, h->G.n / 32 + 1), TPB, 0, s>>>(c));
    CK(cudaGetLastError());
    return MSC_OK;
}

struct FixResult {
    uint32_t n_c = 0, n_s = 0, n_fb = 0;
    std::vector<msc_iter_record> trace;
};

constexpr int GRAPH_ROUNDS = 16;   // C-pass rounds queued per graph launch
constexpr int BATCH_STREAMS = 8;   // jobs of a batch that run at once, one stream each

// A captured graph of GRAPH_ROUNDS C-pass rounds.  With profiling, every kernel node sits
// between two event-record nodes; a node pair is counted only if its round ran.
struct RoundGraph {
    cudaGraphExec_t exec = nullptr;
    struct Pair {
        cudaEvent_t a, b;
        int cls, round, pre;   // pre: the targeting pass and decision, which also run in the
    };                         // round that finds no false case
    std::vector<Pair> pairs;
    ~RoundGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto &p : pairs) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    }
};

// small: one block per SM for every kernel (rounds that edit few vertices, where a launch's
// cost is mostly its blocks starting and finding little to do); otherwise one full wave
template <int D>
msc_status build_round_graph(msc_handle *h, const Ctx &c, unsigned prof_mask, bool small, RoundGraph &rg)
{
    cudaStream_t cs = h->cap_stream;
    cudaGraph_t graph = nullptr;
    // grid sizes (occupancy queries) before the capture begins
    auto grid = [&](const void *k, unsigned long long n) { return small ? std::min(sm_count(), grid_occ(k, n)) : grid_occ(k, n); };
    const int g_ct = grid((const void *)k_ctargets<D>, h->G.n / 8 + 1);
    const int g_tl = grid((const void *)k_tlist, h->G.n / 32 + 1);
    Ctx cm = c;          // the graph's C-pass marks T bits only; k_tlist lists them
    cm.mark_only = 1;
    const int g_ed = grid((const void *)k_edit<D>, h->G.n);
    const int g_mk = grid((const void *)k_mark<D>, 32ull * h->G.n);
    const int g_rf = grid((const void *)k_refresh<D>, h->G.n);
    const int g_rb = grid((const void *)k_rebuild<D>, h->G.n);
    const int g_cl = grid((const void *)k_clear, h->G.n);
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    auto node = [&](int cls, int round, int pre, auto &&launch) {
        if (!((prof_mask >> cls) & 1u)) { launch(); return; }
        RoundGraph::Pair p{nullptr, nullptr, cls, round, pre};
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        cudaEventRecordWithFlags(p.a, cs, cudaEventRecordExternal);   // an event-record node
        launch();
        cudaEventRecordWithFlags(p.b, cs, cudaEventRecordExternal);
        rg.pairs.push_back(p);
    };
    for (int r = 0; r < GRAPH_ROUNDS; r++) {
        node(MSC_K_CPASS, r, 1, [&] { k_ctargets<D><<<g_ct, TPB, 0, cs>>>(cm); });
        node(MSC_K_CPASS, r, 1, [&] { k_tlist<<<g_tl, TPB, 0, cs>>>(cm); });
        node(MSC_K_OTHER, r, 1, [&] { k_decide<<<1, 32, 0, cs>>>(c, 0); });
        node(MSC_K_EDIT, r, 0, [&] { k_edit<D><<<g_ed, TPB, 0, cs>>>(c); });
        node(MSC_K_EDIT, r, 0, [&] { k_mark<D><<<g_mk, TPB, 0, cs>>>(c); });
        node(MSC_K_REFRESH, r, 0, [&] { k_refresh<D><<<g_rf, TPB, 0, cs>>>(c); });
        node(MSC_K_REBUILD, r, 0, [&] { k_rebuild<D><<<g_rb, TPB, 0, cs>>>(c); });
        node(MSC_K_REBUILD, r, 0, [&] { k_clear<<<g_cl, TPB, 0, cs>>>(c); });
        node(MSC_K_OTHER, r, 0, [&] { k_end<<<1, 32, 0, cs>>>(c); });
    }
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (e != cudaSuccess) return fail(MSC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&rg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MSC_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    return MSC_OK;
}

// launch counts (always) and event times (profiling) of one graph launch in which `active`
// rounds edited and `halted` tells whether a further round found no false case
void account_graph(msc_handle *h, RoundGraph &rg, unsigned active, bool halted)
{
    const unsigned long long a = active, t = active + (halted ? 1 : 0);
    h->launches[MSC_K_CPASS] += 2 * t;
    h->launches[MSC_K_OTHER] += t + a;
    h->launches[MSC_K_EDIT] += 2 * a;
    h->launches[MSC_K_REFRESH] += a;
    h->launches[MSC_K_REBUILD] += 2 * a;
    for (auto &p : rg.pairs) {
        const bool ran = (unsigned)p.round < active || ((unsigned)p.round == active && halted && p.pre);
        if (!ran) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            h->ms[p.cls] += ms;
            h->timed[p.cls]++;
        }
    }
    cudaGetLastError();
}

// blocks of the cluster form of the round kernel on the current device: 16 where a cluster
// of that size can be resident (a size beyond the portable 8), else 8, else 0 (no cluster form)
template <int D> int round_cluster_size()
{
    static std::mutex mu;
    static std::map<int, int> by_dev;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
    std::lock_guard<std::mutex> lk(mu);
    auto it = by_dev.find(dev);
    if (it != by_dev.end()) return it->second;
    int best = 0;
    if (cudaFuncSetAttribute(k_rounds<D, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int cs : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)cs);
        cfg.blockDim = dim3(TPB);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_rounds<D, true>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        if (n >= 1) { best = cs; break; }
    }
    by_dev[dev] = best;
    return best;
}

template <int D>
msc_status fix_loop(msc_handle *h, float xi, const msc_options &o, cudaStream_t s, FixResult &R)
{
    Ctx c = make_ctx(h, o.tier, o.q_max, o.exact_fallback, xi, o.edit_mode);
    LoopState L{};
    L.max_iters = (unsigned)o.max_iters;
    L.exact_fallback = (unsigned)o.exact_fallback;
    if (o.record_trace) {
        L.trace_cap = (unsigned)std::min<long long>(std::max(o.max_iters, 1), 1 << 22);
        CK(h->trace.alloc(6ull * L.trace_cap));
        c.trace = h->trace.p;
    }
    // rounds that edit few vertices run in the persistent kernel when the device has
    // cooperative launches, else in a graph of small grids
    int rgrid = h->rounds_grid > 0 ? h->rounds_grid : sm_count();
    {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)k_rounds<D, false>, TPB, 0) != cudaSuccess) {
            cudaGetLastError();
            occ = 0;
        }
        rgrid = std::min(rgrid, occ * sm_count());
    }
    const bool persistent = coop_supported() && rgrid > 0;
    L.rounds_kernel = persistent ? 1 : 0;
    const unsigned long long small_thr = o.small_round > 0 ? (unsigned long long)o.small_round : SMALL_ROUND;
    // the rounds after one that edited fewer than clus_thr vertices run in one cluster
    const unsigned long long clus_thr = o.cluster_round > 0 ? (unsigned long long)o.cluster_round : CLUSTER_ROUND;
    const int csize = persistent && o.cluster_round != 1 ? round_cluster_size<D>() : 0;
    L.small_round = small_thr;
    CK(cudaMemcpyAsync(h->ls.p, &L, sizeof L, cudaMemcpyHostToDevice, s));
    KL(h, MSC_K_OTHER, s, k_init_g<<<grid_occ((const void *)k_init_g, h->G.n), TPB, 0, s>>>(h->f.p, h->fhat.p, h->g.p, h->gprev.p, h->state.p, h->G.n, xi));
    CK(cudaGetLastError());
    // sets left over by an earlier call that stopped with an error
    CK(cudaMemsetAsync(h->Tbits.p, 0, h->Tbits.n * 4, s));
    CK(cudaMemsetAsync(h->Xbits.p, 0, h->Xbits.n * 4, s));
    CK(cudaMemsetAsync(h->Dbits.p, 0, h->Dbits.n * 4, s));
    CK(cudaMemsetAsync(h->sDbits.p, 0, h->sDbits.n * 4, s));
    CK(cudaMemsetAsync(h->cnt.p, 0, sizeof(Counters), s));
    LoopState *ls = h->ls.p;
    CK(cudaMemsetAsync(h->Csum.p, 0, h->Csum.n * 4, s));
    CKS(eval_dense<D>(h, h->g.p, h->G, h->code_g.p, s, h->code_f.p, h->Mbits.p, h->Cbits.p, h->Csum.p, o.tier));
    KL(h, MSC_K_REBUILD, s, k_list_blocks<<<grid_occ((const void *)k_list_blocks, h->G.n / 1024 + 1), TPB, 0, s>>>(c));
    h->items[MSC_K_DENSE] += h->G.n;
    // two captured graphs: full grids for rounds that edit many vertices, one block per SM
    // for the long tail of rounds that edit few (chosen by the last round's size)
    RoundGraph rg_big, rg_small;
    CKS(build_round_graph<D>(h, c, (unsigned)o.profile & MSC_PROFILE_ALL, false, rg_big));
    if (!persistent) CKS(build_round_graph<D>(h, c, (unsigned)o.profile & MSC_PROFILE_ALL, true, rg_small));
    bool sep_built = false;
    unsigned prev_iters = 0;
    unsigned long long fix_work[3] = {0, 0, 0};   // items of this call done by the round kernel
    for (;;) {
        if (g_cancel && g_cancel->load()) return fail(MSC_ERR_CANCELLED, "the job was cancelled");
        const bool small = L.iters > 0 && L.last_items < small_thr;
        if (small && persistent) {
            const LoopState L0 = L;
            KL(h, MSC_K_OTHER, s, k_rounds_enter<<<1, 1, 0, s>>>(ls, h->bar.p));
            CK(cudaMemsetAsync(h->cnt.p, 0, 2 * sizeof(Counters), s));
            Counters *cnt2 = h->cnt.p;
            uint32_t *blk2 = h->Cblk2.p;
            GridBarrier *gb = h->bar.p;
            unsigned max_rounds = 1u << 30;
            // the cluster form's C-pass: up to two listed blocks per warp
            unsigned long long blk_limit = 2ull * (unsigned long long)csize * (TPB / 32);
            const bool tiny = csize > 0 && L.last_items < clus_thr && L.nblk <= blk_limit;
            unsigned long long leave = tiny ? clus_thr : small_thr, below = !tiny && csize > 0 ? clus_thr : 0;
            cudaError_t le = cudaSuccess;
            if (tiny) {
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)csize;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3((unsigned)csize);
                cfg.blockDim = dim3(TPB);
                cfg.stream = s;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                KL(h, MSC_K_ROUNDS, s, le = cudaLaunchKernelEx(&cfg, k_rounds<D, true>, c, gb, cnt2, blk2, max_rounds, leave, below,
                                                                blk_limit));
            } else {
                void *args[] = {(void *)&c, (void *)&gb, (void *)&cnt2, (void *)&blk2, (void *)&max_rounds, (void *)&leave,
                                (void *)&below, (void *)&blk_limit};
                KL(h, MSC_K_ROUNDS, s, le = cudaLaunchCooperativeKernel((const void *)k_rounds<D, false>, dim3(rgrid), dim3(TPB), args, 0, s));
            }
            if (le != cudaSuccess) return fail(MSC_ERR_CUDA, "persistent round kernel launch failed: %s", cudaGetErrorString(le));
            KL(h, MSC_K_OTHER, s, k_rounds_leave<<<1, 1, 0, s>>>(ls));
            KL(h, MSC_K_REBUILD, s, k_list_blocks<<<grid_occ((const void *)k_list_blocks, h->G.n / 1024 + 1), TPB, 0, s>>>(c));
            CK(cudaMemsetAsync(h->cnt.p, 0, sizeof(Counters), s));
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(&L, ls, sizeof L, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            prev_iters = L.iters;
            h->items[MSC_K_ROUNDS] += L.iters - L0.iters;
            if (tiny) {
                h->cluster_launches++;
                h->cluster_rounds += L.iters - L0.iters;
            }
            for (int q = 0; q < 4; q++) h->round_phase_ns[q] += L.phase_ns[q] - L0.phase_ns[q];
            fix_work[0] += L.edit_items - L0.edit_items;
            fix_work[1] += L.refresh_items - L0.refresh_items;
            fix_work[2] += L.cpass_items - L0.cpass_items;
            if (L.status == MSC_ERR_DEVICE_TIMEOUT)
                return fail(MSC_ERR_DEVICE_TIMEOUT, "a grid barrier of the persistent round kernel timed out");
        } else {
            RoundGraph &rg = small ? rg_small : rg_big;
            if (L.leave) KL(h, MSC_K_OTHER, s, k_set_leave<<<1, 1, 0, s>>>(ls, 0));
            CK(cudaGraphLaunch(rg.exec, s));
            CK(cudaMemcpyAsync(&L, ls, sizeof L, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            account_graph(h, rg, L.iters - prev_iters, L.halt != 0);
            prev_iters = L.iters;
        }
        if (L.status == MSC_ERR_STALLED)
            return fail(MSC_ERR_STALLED, "every false case targets a vertex that can no longer move");
        if (L.status == MSC_ERR_NOT_CONVERGED) return fail(MSC_ERR_NOT_CONVERGED, "not converged after %d edit rounds", o.max_iters);
        if (!L.halt) continue;               // the C-pass phase goes on
        if (o.tier < 3) break;
        // S-pass (Sec. 4.4) on the current lists
        CK(cudaMemsetAsync(h->cnt.p, 0, sizeof(Counters), s));
        const bool first_build = o.tier >= 4 && !sep_built;
        if (o.tier >= 4) CKS(s_pass_state<D>(h, c, sep_built, &ls->nSD, s));
        else CKS(s_pass<D>(h, c, o.tier, s));
        Counters hc;
        CK(cudaMemcpyAsync(&hc, h->cnt.p, sizeof hc, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        h->items[first_build ? MSC_K_SEP_SEED : MSC_K_SEP_UPDATE] += hc.steps[0] + hc.steps[1] + hc.steps[2];
        if (hc.err) return fail(MSC_ERR_OOM, "separatrix spill queue overflow");
        if (hc.ncase == 0) break;
        // the S-pass edit round, then back to C-pass rounds
        KL(h, MSC_K_OTHER, s, k_set_halt<<<1, 1, 0, s>>>(ls, 0));
        KL(h, MSC_K_OTHER, s, k_set_leave<<<1, 1, 0, s>>>(ls, 0));
        KL(h, MSC_K_OTHER, s, k_decide<<<1, 32, 0, s>>>(c, 1));
        KL(h, MSC_K_EDIT, s, k_edit<D><<<grid_occ((const void *)k_edit<D>, h->G.n), TPB, 0, s>>>(c));
        KL(h, MSC_K_EDIT, s, k_mark<D><<<grid_occ((const void *)k_mark<D>, 32ull * h->G.n), TPB, 0, s>>>(c));
        KL(h, MSC_K_REFRESH, s, k_refresh<D><<<grid_occ((const void *)k_refresh<D>, h->G.n), TPB, 0, s>>>(c));
        KL(h, MSC_K_REBUILD, s, k_rebuild<D><<<grid_occ((const void *)k_rebuild<D>, h->G.n), TPB, 0, s>>>(c));
        KL(h, MSC_K_REBUILD, s, k_clear<<<grid_occ((const void *)k_clear, h->G.n), TPB, 0, s>>>(c));
        KL(h, MSC_K_OTHER, s, k_end<<<1, 32, 0, s>>>(c));
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&L, ls, sizeof L, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        prev_iters = L.iters;
        if (L.status == MSC_ERR_STALLED)
            return fail(MSC_ERR_STALLED, "every false case targets a vertex that can no longer move");
        if (L.status == MSC_ERR_NOT_CONVERGED) return fail(MSC_ERR_NOT_CONVERGED, "not converged after %d edit rounds", o.max_iters);
    }
    R.n_c = L.n_c;
    R.n_s = L.n_s;
    R.n_fb = L.n_fb;
    h->items[MSC_K_EDIT] += L.edit_items - fix_work[0];
    h->items[MSC_K_REFRESH] += L.refresh_items - fix_work[1];
    h->items[MSC_K_CPASS] += L.cpass_items - fix_work[2];
    h->items[MSC_K_REBUILD] += L.refresh_items - fix_work[1];
    for (int i = 0; i < 3; i++) h->round_work[i] += fix_work[i];
    if (o.record_trace && L.ntrace) {
        const unsigned nt = std::min(L.ntrace, L.trace_cap);
        std::vector<int64_t> rows(6ull * nt);
        CK(cudaMemcpyAsync(rows.data(), h->trace.p, rows.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (unsigned i = 0; i < nt; i++) {
            msc_iter_record r{};
            r.kind = (int32_t)rows[6 * i];
            r.t_us = (int32_t)std::min<int64_t>((rows[6 * i + 5] - rows[5]) / 1000, INT32_MAX);
            r.n_targets = rows[6 * i + 1];
            r.n_exact = rows[6 * i + 2];
            r.sum_targets = rows[6 * i + 3];
            r.sum_exact = rows[6 * i + 4];
            R.trace.push_back(r);
        }
    }
    return MSC_OK;
}

msc_status write_edits(msc_handle *h, float xi, int qmax, cudaStream_t s, msc_edits *out)
{
    const uint32_t n = h->G.n;
    const uint32_t nb = (n + 1023) / 1024;
    DevBuf<uint8_t> qm;
    DevBuf<uint32_t> bc;
    DevBuf<unsigned long long> tot;
    CK(qm.alloc(n));
    CK(bc.alloc(nb));
    CK(tot.alloc(2));
    CK(cudaMemsetAsync(tot.p, 0, 2 * sizeof(unsigned long long), s));
    KL(h, MSC_K_OTHER, s, k_qmap<<<nb, 1024, 0, s>>>(h->f.p, h->fhat.p, h->state.p, n, xi, qmax, qm.p, bc.p, tot.p + 1));
    KL(h, MSC_K_OTHER, s, k_scan_blocks<<<1, 1024, 0, s>>>(bc.p, nb, tot.p));
    CK(cudaGetLastError());
    unsigned long long t[2];
    CK(cudaMemcpyAsync(t, tot.p, sizeof t, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    DevBuf<uint64_t> li;
    DevBuf<float> lv;
    CK(li.alloc(t[0]));
    CK(lv.alloc(t[0]));
    KL(h, MSC_K_OTHER, s, k_lossless_write<<<nb, 1024, 0, s>>>(qm.p, h->g.p, n, bc.p, li.p, lv.p));
    CK(cudaGetLastError());
    out->n_vertices = n;
    out->n_lossless = t[0];
    out->n_quant = t[1];
    out->q_map = (uint8_t *)host_take(n ? n : 1);
    out->lossless_idx = (uint64_t *)host_take(t[0] ? t[0] * 8 : 8);
    out->lossless_val = (float *)host_take(t[0] ? t[0] * 4 : 4);
    if (!out->q_map || !out->lossless_idx || !out->lossless_val) return fail(MSC_ERR_OOM, "host allocation of edits failed");
    CK(cudaMemcpyAsync(out->q_map, qm.p, n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->lossless_idx, li.p, t[0] * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(out->lossless_val, lv.p, t[0] * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MSC_OK;
}

template <int D> msc_status verify_impl(msc_handle *h, const float *gdev, float xi, cudaStream_t s, msc_report *out)
{
    DevBuf<uint64_t> code;
    CK(code.alloc(h->G.n));
    CKS(eval_dense<D>(h, gdev, h->G, code.p, s));
    CK(cudaMemsetAsync(h->cnt.p, 0, sizeof(Counters), s));
    KL(h, MSC_K_OTHER, s, k_decode_crit<D><<<grid_occ((const void *)k_decode_crit<D>, h->G.n), TPB, 0, s>>>(code.p, h->code_f.p, h->G, nullptr, nullptr, nullptr, 0, h->cnt.p));
    KL(h, MSC_K_OTHER, s, k_max_abs_err<<<grid_occ((const void *)k_max_abs_err, h->G.n), TPB, 0, s>>>(h->f.p, gdev, h->G.n, &h->cnt.p->rep[13]));
    CK(cudaGetLastError());
    Counters hc;
    CK(cudaMemcpyAsync(&hc, h->cnt.p, sizeof hc, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memset(out, 0, sizeof *out);
    unsigned long long crit_bad = 0;
    for (int d = 0; d < 4; d++) {
        out->fp[d] = hc.rep[d];
        out->fn[d] = hc.rep[4 + d];
        crit_bad += hc.rep[d] + hc.rep[4 + d];
    }
    double m;
    memcpy(&m, &hc.rep[13], sizeof m);
    out->max_abs_err = m;
    if (crit_bad == 0) {
        Ctx c = make_ctx(h, 4, 6, 0, xi);
        c.g = (float *)gdev;
        c.code_g = code.p;
        // per-separatrix pair and end checks
        CK(cudaMemsetAsync(h->cnt.p, 0, sizeof(Counters), s));
        if (h->n_desc) KL(h, MSC_K_OTHER, s, k_verify_desc<D><<<grid_occ((const void *)k_verify_desc<D>, h->n_desc), TPB, 0, s>>>(c, h->seeds_desc.p, h->n_desc));
        if (h->n_asc) KL(h, MSC_K_OTHER, s, k_verify_asc<D><<<grid_occ((const void *)k_verify_asc<D>, h->n_asc), TPB, 0, s>>>(c, h->seeds_asc.p, h->n_asc));
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&hc, h->cnt.p, sizeof hc, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        out->sep_mismatch[0] = hc.rep[8];
        out->sep_mismatch[1] = hc.rep[9];
        out->term_mismatch[0] = hc.rep[11];
        out->term_mismatch[1] = hc.rep[12];
        if (D == 3) {
            // saddle-saddle connectors: troublemakers found by the tier-4 walk (count only)
            DevBuf<uint32_t> tl, tb, xl, xb;
            CK(tl.alloc(h->G.n)); CK(tb.alloc(words(h->G.n)));
            CK(xl.alloc(1)); CK(xb.alloc(words(h->G.n)));
            CK(cudaMemsetAsync(tb.p, 0, tb.n * 4, s));
            CK(cudaMemsetAsync(xb.p, 0, xb.n * 4, s));
            DevBuf<uint8_t> st;
            CK(st.alloc(h->G.n));
            CK(cudaMemsetAsync(st.p, 0, h->G.n, s));
            // per 2-saddle: the walk marks the triangles whose facets hold a troublemaker,
            // then backward steps mark every reached triangle that leads to one
            DevBuf<uint32_t> bad, bl0, bl1;
            DevBuf<unsigned long long> bn;
            const uint32_t bcap = (uint32_t)h->G.n + 1;
            CK(bad.alloc(words(h->G.n * 12))); CK(bl0.alloc(bcap)); CK(bl1.alloc(bcap)); CK(bn.alloc(4));
            CK(cudaMemsetAsync(bad.p, 0, bad.n * 4, s));
            CK(cudaMemsetAsync(bn.p, 0, 4 * sizeof(unsigned long long), s));
            Ctx v = c;
            v.Tlist = tl.p; v.Tbits = tb.p; v.Xlist = xl.p; v.Xbits = xb.p; v.state = st.p;
            v.exact_fallback = 0;
            v.ss_bad = bad.p; v.ss_list = bl0.p; v.ss_n = bn.p; v.ss_cap = bcap;
            CK(cudaMemsetAsync(h->cnt.p, 0, sizeof(Counters), s));
            CK(cudaMemsetAsync(h->vis_tri.p, 0, h->vis_tri.n * 4, s));
            v.ovf_out = h->ovf0.p;
            if (h->n_ss) KL(h, MSC_K_SEP_UPDATE, s, k_ss_seed<<<grid_occ((const void *)k_ss_seed, h->n_ss), TPB, 0, s>>>(v, h->seeds_ss.p, h->n_ss));
            CK(cudaGetLastError());
            uint32_t *in = h->ovf0.p, *o2 = h->ovf1.p;
            for (;;) {
                CK(cudaMemcpyAsync(&hc, h->cnt.p, sizeof hc, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (hc.err) return fail(MSC_ERR_OOM, "saddle-saddle spill queue overflow");
                if (hc.novf == 0) break;
                const unsigned long long zero = 0;
                CK(cudaMemcpyAsync(&h->cnt.p->novf, &zero, sizeof zero, cudaMemcpyHostToDevice, s));
                v.ovf_out = o2;
                KL(h, MSC_K_SEP_UPDATE, s, k_ss_spill<<<grid_occ((const void *)k_ss_spill, hc.novf), TPB, 0, s>>>(v, in, (uint32_t)hc.novf));
                CK(cudaGetLastError());
                std::swap(in, o2);
            }
            uint32_t *bin = bl0.p, *bout = bl1.p;
            for (int side = 0;; side ^= 1) {
                unsigned long long nb[4];
                CK(cudaMemcpyAsync(nb, bn.p, sizeof nb, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                unsigned long long err = 0;
                CK(cudaMemcpyAsync(&err, &h->cnt.p->err, sizeof err, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (err) return fail(MSC_ERR_OOM, "saddle-saddle verification list overflow");
                const unsigned long long m = nb[side];
                if (m == 0) break;
                CK(cudaMemsetAsync(bn.p + (side ^ 1), 0, sizeof(unsigned long long), s));
                KL(h, MSC_K_OTHER, s, k_ss_back<<<grid_occ((const void *)k_ss_back, m), TPB, 0, s>>>(v, bin, (uint32_t)m, bout, bn.p + (side ^ 1), bcap));
                CK(cudaGetLastError());
                CK(cudaMemsetAsync(bn.p + side, 0, sizeof(unsigned long long), s));
                std::swap(bin, bout);
            }
            CK(cudaMemsetAsync(bn.p + 2, 0, sizeof(unsigned long long), s));
            if (h->n_ss) KL(h, MSC_K_OTHER, s, k_ss_count<<<grid_occ((const void *)k_ss_count, h->n_ss), TPB, 0, s>>>(v, h->seeds_ss.p, h->n_ss, bn.p + 2));
            CK(cudaGetLastError());
            unsigned long long nbad = 0;
            CK(cudaMemcpyAsync(&nbad, bn.p + 2, sizeof nbad, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            out->sep_mismatch[2] = nbad;
        }
    }
    unsigned long long sep = 0;
    for (int i = 0; i < 3; i++) sep += out->sep_mismatch[i];
    const bool bound = out->max_abs_err <= (double)xi;
    const bool ext = out->fp[0] + out->fn[0] + out->fp[D] + out->fn[D] == 0;
    const bool term = out->term_mismatch[0] + out->term_mismatch[1] == 0;
    out->pass_tier[0] = bound && ext;
    out->pass_tier[1] = bound && crit_bad == 0;
    out->pass_tier[2] = out->pass_tier[1] && term;
    out->pass_tier[3] = out->pass_tier[2] && sep == 0;
    out->pass = out->pass_tier[3];
    return MSC_OK;
}

// a device copy of a caller's field (owned here only if the caller passed host memory)
struct DevInput {
    DevBuf<float> own;
    const float *p = nullptr;
};

msc_status device_input(const float *src, size_t n, DevInput &d, cudaStream_t s, const char *what)
{
    if (!src) return fail(MSC_ERR_INVALID_ARG, "%s is NULL", what);
    if (is_device_ptr(src)) { d.p = src; return MSC_OK; }
    CK(d.own.alloc(n));
    CK(copy_to_device(d.own.p, src, n * sizeof(float), s));
    d.p = d.own.p;
    return MSC_OK;
}

template <int D>
msc_status introspect(const float *field, Grid G, int what, int64_t *rows, int32_t *dims, uint64_t cap, uint64_t *n_out)
{
    cudaStream_t s = nullptr;
    DevBuf<float> v;
    DevBuf<uint64_t> code;
    DevBuf<unsigned long long> cnt;
    CK(v.alloc(G.n));
    CK(code.alloc(G.n));
    CK(cnt.alloc(2));
    CKS(upload_field(nullptr, field, G.n, v.p, cnt.p, s, "field"));
    CKS(eval_dense<D>(nullptr, v.p, G, code.p, s));
    CK(cudaMemsetAsync(cnt.p, 0, 8, s));
    if (what == 0) k_decode_pairs<D><<<grid_occ((const void *)k_decode_pairs<D>, G.n), TPB, 0, s>>>(code.p, G, nullptr, cnt.p, 0);
    else k_decode_crit<D><<<grid_occ((const void *)k_decode_crit<D>, G.n), TPB, 0, s>>>(code.p, nullptr, G, nullptr, nullptr, cnt.p, 0, nullptr);
    CK(cudaGetLastError());
    unsigned long long n = 0;
    CK(cudaMemcpy(&n, cnt.p, 8, cudaMemcpyDeviceToHost));
    *n_out = n;
    if (!cap || !rows) return MSC_OK;
    const unsigned long long m = n < cap ? n : cap;
    const int w = what == 0 ? 8 : 4;
    DevBuf<int64_t> r;
    DevBuf<int32_t> dd;
    CK(r.alloc(m * w));
    CK(dd.alloc(m));
    CK(cudaMemsetAsync(cnt.p, 0, 8, s));
    if (what == 0) k_decode_pairs<D><<<grid_occ((const void *)k_decode_pairs<D>, G.n), TPB, 0, s>>>(code.p, G, r.p, cnt.p, m);
    else k_decode_crit<D><<<grid_occ((const void *)k_decode_crit<D>, G.n), TPB, 0, s>>>(code.p, nullptr, G, r.p, dd.p, cnt.p, m, nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpy(rows, r.p, m * w * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (what == 1 && dims) CK(cudaMemcpy(dims, dd.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return MSC_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------
// packed edit record (Sec. 4.7)
// ------------------------------------------------------------------------------------
namespace {
int pack_bits(int qmax)
{
    int b = 1;
    while ((1 << b) < qmax + 2) b++;
    return b;
}

uint64_t packed_size(uint64_t n, uint64_t nl, int qmax) { return 32 + ((n + 7) / 8) * pack_bits(qmax) + 4 * nl; }

void put_u64(uint8_t *p, uint64_t v)
{
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}

uint64_t get_u64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

// bytes between host and/or device buffers
cudaMemcpyKind copy_kind(const void *dst, const void *src)
{
    const bool dd = is_device_ptr(dst), sd = is_device_ptr(src);
    return dd ? (sd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice) : (sd ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
}

// the lossless positions of a device q-map in increasing order (idx, device), their number,
// and the number of quantised (non-zero) counts; counts above q_max are an error
msc_status lossless_positions(const uint8_t *qm, uint64_t n, int qmax, DevBuf<uint64_t> &idx, uint64_t *nl,
                              uint64_t *nq, cudaStream_t s)
{
    const uint32_t nb = (uint32_t)((n + 1023) / 1024);
    DevBuf<uint32_t> bc;
    DevBuf<unsigned long long> tot;
    CK(bc.alloc(nb));
    CK(tot.alloc(3));
    CK(cudaMemsetAsync(tot.p, 0, 3 * sizeof(unsigned long long), s));
    k_qcount<<<nb, 1024, 0, s>>>(qm, n, qmax, bc.p, tot.p + 1, tot.p + 2);
    k_scan_blocks<<<1, 1024, 0, s>>>(bc.p, nb, tot.p);
    CK(cudaGetLastError());
    unsigned long long t[3];
    CK(cudaMemcpyAsync(t, tot.p, sizeof t, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (t[2]) return fail(MSC_ERR_INVALID_ARG, "q-map holds %llu counts above q_max = %d", t[2], qmax);
    CK(idx.alloc(t[0]));
    k_lossless_write<<<nb, 1024, 0, s>>>(qm, nullptr, (uint32_t)n, bc.p, idx.p, nullptr);
    CK(cudaGetLastError());
    *nl = t[0];
    *nq = t[1];
    return MSC_OK;
}
}  // namespace

// ------------------------------------------------------------------------------------
// fixed scratch of msc_critical_cells_static: gradient codes of up to
// MSC_STATIC_MAX_VERTICES anchors, then [0] the row count, [1] the non-finite count
// ------------------------------------------------------------------------------------
namespace {
constexpr size_t STATIC_WORDS = (size_t)MSC_STATIC_MAX_VERTICES + 32;
}
static __device__ __align__(256) unsigned long long g_static_scratch[STATIC_WORDS];

namespace {
// device address of the static scratch on the current device.  Looked up on every call:
// the lookup is cheap, and an address kept from an earlier call would be stale after the
// device's context was torn down and the module loaded again.
msc_status static_scratch(unsigned long long **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(MSC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    }
    *out = (unsigned long long *)p;
    return MSC_OK;
}

// true iff p is device memory of the current device, or managed memory
bool on_current_device(const void *p)
{
    cudaPointerAttributes a;
    int dev = -1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

template <int D>
msc_status critical_static(const float *field, Grid G, int64_t *rows, int32_t *dims, uint64_t cap, uint64_t *n_out,
                           cudaStream_t s)
{
    unsigned long long *scr = nullptr;
    CKS(static_scratch(&scr));
    // waits for the stream on every return path, so that no kernel of this call is still
    // writing the scratch or the caller's rows when it returns
    struct SyncOnExit {
        cudaStream_t s;
        ~SyncOnExit()
        {
            cudaStreamSynchronize(s);
            cudaGetLastError();
        }
    } sync_on_exit{s};
    uint64_t *code = (uint64_t *)scr;
    unsigned long long *count = scr + MSC_STATIC_MAX_VERTICES, *bad = count + 1;
    CK(cudaMemsetAsync(count, 0, 2 * sizeof(unsigned long long), s));
    k_count_nonfinite<<<grid_occ((const void *)k_count_nonfinite, G.n), TPB, 0, s>>>(field, G.n, bad);
    k_eval_dense<D><<<grid_occ((const void *)k_eval_dense<D>, G.n), TPB, 0, s>>>(field, G, code, nullptr, nullptr, nullptr, nullptr, 4);
    k_decode_crit<D><<<grid_occ((const void *)k_decode_crit<D>, G.n), TPB, 0, s>>>(code, nullptr, G, cap ? rows : nullptr, dims, count, cap, nullptr);
    CK(cudaGetLastError());
    unsigned long long hv[2];
    CK(cudaMemcpyAsync(hv, count, sizeof hv, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hv[1]) return fail(MSC_ERR_INVALID_ARG, "field has %llu non-finite values", hv[1]);
    *n_out = hv[0];
    return MSC_OK;
}
}  // namespace

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
void msc_rt::limit_cached_memory(uint64_t bytes)
{
    cudaMemPool_t pool = lib_pool();
    if (pool) cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &bytes);
    cudaGetLastError();
}

void msc_rt::set_cancel_flag(const std::atomic<int> *flag) { g_cancel = flag; }

void msc_rt::share_device(msc_handle *h, int concurrent)
{
    if (h && concurrent > 1) h->rounds_grid = std::max(16, 2 * sm_count() / concurrent);
}

extern "C" {

const char *msc_version(void) { return "msc-gb300 0.1 (sm_103a)"; }

const char *msc_status_string(msc_status s)
{
    switch (s) {
    case MSC_OK: return "MSC_OK";
    case MSC_ERR_INVALID_ARG: return "MSC_ERR_INVALID_ARG";
    case MSC_ERR_OOM: return "MSC_ERR_OOM";
    case MSC_ERR_CUDA: return "MSC_ERR_CUDA";
    case MSC_ERR_CANCELLED: return "MSC_ERR_CANCELLED";
    case MSC_ERR_UNAVAILABLE: return "MSC_ERR_UNAVAILABLE";
    case MSC_ERR_NOT_CONVERGED: return "MSC_ERR_NOT_CONVERGED";
    case MSC_ERR_DEVICE_TIMEOUT: return "MSC_ERR_DEVICE_TIMEOUT";
    case MSC_ERR_STALLED: return "MSC_ERR_STALLED";
    case MSC_ERR_NO_DEVICE: return "MSC_ERR_NO_DEVICE";
    }
    return "MSC_ERR_UNKNOWN";
}

const char *msc_last_error(void) { return g_last_error.c_str(); }

void msc_default_options(msc_options *opt)
{
    if (opt) fill_defaults(opt);
}

uint64_t msc_device_bytes(int nx, int ny, int nz)
{
    const uint64_t n = (uint64_t)nx * ny * nz;
    const bool d3 = nz > 1;
    const uint64_t ntop = d3 ? 6 : 2;
    uint64_t b = 12 * n + n + 16 * n;             // f, f_hat, g; state; code_f, code_g
    b += 4 * (n / 8 + 4) + 8 * 4 * n;             // four bitsets; eight index lists
    b += n / 8 + ntop * n / 8 + (d3 ? 12 * n / 8 + 16 * ovf_pairs(n) : 0);   // walk visited sets, spill queues
    b += 2 * n * (1 + ntop + (d3 ? 19 : 0));      // separatrix node words (16 bits each)
    b += (d3 ? 6 : 3) * 4 * n;                    // separatrix seeds (upper estimate)
    b += 8 * n;                                   // pre-round values and list of edited vertices
    return b;
}

msc_status msc_prepare_original(const float *f, int nx, int ny, int nz, const msc_options *opt, msc_handle **out)
{
    g_last_error.clear();
    if (!out) return fail(MSC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    CKS(check_dims(nx, ny, nz));
    msc_options o;
    if (opt) o = *opt; else fill_defaults(&o);
    CKS(check_options(&o));
    CKS(device_ready());
    cudaStream_t s = (cudaStream_t)o.stream;
    EntryStream es(s);
    msc_handle *h = new (std::nothrow) msc_handle();
    if (!h) return fail(MSC_ERR_OOM, "handle allocation failed");
    h->G = make_grid(nx, ny, nz);
    h->D = nz > 1 ? 3 : 2;
    {
        const msc_status ts = tile_request(o, &h->tile_req);
        if (ts != MSC_OK) { delete h; return ts; }
    }
    auto run = [&]() -> msc_status {
        CK(h->f.alloc(h->G.n));
        CK(h->code_f.alloc(h->G.n));
        if (h->D == 3) CK(h->low_f.alloc(h->G.n));
        CK(h->cnt.alloc(1));
        CK(h->nM.alloc(8));
        h->prof_mask = (unsigned)o.profile & MSC_PROFILE_ALL;
        CKS(upload_field(h, f, h->G.n, h->f.p, h->nM.p, s, "f"));
        if (h->D == 3) CK(h->seed_count.alloc(3));
        CKS(eval_dense_any(h, h->D, h->f.p, h->G, h->code_f.p, s, h->D == 3 ? h->low_f.p : nullptr));
        h->items[MSC_K_DENSE] += h->G.n;
        CKS(h->D == 3 ? build_seeds<3>(h, s) : build_seeds<2>(h, s));
        CK(cudaEventCreate(&h->ev0));
        CK(cudaEventCreate(&h->ev1));
        CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamSynchronize(s));
        prof_flush(h);
        h->prof_mask = 0;
        return MSC_OK;
    };
    msc_status st = run();
    if (st != MSC_OK) { msc_destroy(h); return st; }
    *out = h;
    return MSC_OK;
}

msc_status msc_fix(msc_handle *h, const float *f_hat, float xi, const msc_options *opt, msc_edits *out, float *g_out)
{
    g_last_error.clear();
    if (!h || !out || !g_out) return fail(MSC_ERR_INVALID_ARG, "handle, out and g_out must be non-NULL");
    memset(out, 0, sizeof *out);
    msc_options o;
    if (opt) o = *opt; else fill_defaults(&o);
    CKS(check_options(&o));
    if (!(xi > 0.0f) || !std::isfinite(xi)) return fail(MSC_ERR_INVALID_ARG, "xi must be finite and > 0");
    cudaStream_t s = (cudaStream_t)o.stream;
    EntryStream es(s);
    CKS(tile_request(o, &h->tile_req));
    CKS(alloc_fix_state(h));
    h->prof_mask = (unsigned)o.profile & MSC_PROFILE_ALL;
    struct Flush {
        msc_handle *h;
        ~Flush() { prof_flush(h); h->prof_mask = 0; }
    } flush_at_exit{h};
    CKS(upload_field(h, f_hat, h->G.n, h->fhat.p, h->nM.p + 2, s, "f_hat"));
    FixResult R;
    CK(cudaEventRecord(h->ev0, s));
    msc_status st = h->D == 3 ? fix_loop<3>(h, xi, o, s, R) : fix_loop<2>(h, xi, o, s, R);
    if (st != MSC_OK) return st;
    CK(cudaEventRecord(h->ev1, s));
    CK(copy_from_device(g_out, h->g.p, (size_t)h->G.n * 4, s));
    // floating edits: every edited vertex is stored losslessly (state > 0 reads as above a
    // q_max of 0)
    CKS(write_edits(h, xi, o.edit_mode == MSC_EDITS_FLOAT ? 0 : o.q_max, s, out));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    out->loop_ms = ms;
    out->n_iters_c = R.n_c;
    out->n_iters_s = R.n_s;
    out->n_fallback_iters = R.n_fb;
    if (o.record_trace && !R.trace.empty()) {
        out->trace = (msc_iter_record *)malloc(R.trace.size() * sizeof(msc_iter_record));
        if (!out->trace) return fail(MSC_ERR_OOM, "trace allocation failed");
        memcpy(out->trace, R.trace.data(), R.trace.size() * sizeof(msc_iter_record));
        out->n_trace = (uint32_t)R.trace.size();
    }
    return MSC_OK;
}

msc_status msc_apply_edits(const float *f_hat, int nx, int ny, int nz, float xi, int q_max, const msc_edits *e, float *g_out)
{
    g_last_error.clear();
    CKS(check_dims(nx, ny, nz));
    if (!e || !g_out || !e->q_map) return fail(MSC_ERR_INVALID_ARG, "edits and g_out must be non-NULL");
    if (!(xi > 0.0f) || q_max < 1 || q_max > 7) return fail(MSC_ERR_INVALID_ARG, "bad xi or q_max");
    CKS(device_ready());
    const uint32_t n = (uint32_t)((uint64_t)nx * ny * nz);
    if (e->n_vertices != n) return fail(MSC_ERR_INVALID_ARG, "edits are for %llu vertices, grid has %u", (unsigned long long)e->n_vertices, n);
    cudaStream_t s = nullptr;
    EntryStream es(s);
    DevInput fh;
    CKS(device_input(f_hat, n, fh, s, "f_hat"));
    DevBuf<uint8_t> qm;
    DevBuf<uint64_t> li;
    DevBuf<float> lv, g;
    CK(qm.alloc(n));
    CK(li.alloc(e->n_lossless));
    CK(lv.alloc(e->n_lossless));
    CK(g.alloc(n));
    CK(cudaMemcpyAsync(qm.p, e->q_map, n, cudaMemcpyHostToDevice, s));
    if (e->n_lossless) {
        CK(cudaMemcpyAsync(li.p, e->lossless_idx, e->n_lossless * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(lv.p, e->lossless_val, e->n_lossless * 4, cudaMemcpyHostToDevice, s));
    }
    k_apply_q<<<grid_occ((const void *)k_apply_q, n), TPB, 0, s>>>(fh.p, qm.p, n, xi / (float)(1 << q_max), g.p);
    if (e->n_lossless) k_apply_lossless<<<grid_occ((const void *)k_apply_lossless, e->n_lossless), TPB, 0, s>>>(li.p, lv.p, e->n_lossless, g.p);
    CK(cudaGetLastError());
    CK(copy_from_device(g_out, g.p, (size_t)n * 4, s));
    CK(cudaStreamSynchronize(s));
    return MSC_OK;
}

msc_status msc_verify(msc_handle *h, const float *g, float xi, msc_report *out)
{
    g_last_error.clear();
    if (!h || !g || !out) return fail(MSC_ERR_INVALID_ARG, "handle, g and out must be non-NULL");
    if (!(xi > 0.0f)) return fail(MSC_ERR_INVALID_ARG, "xi must be > 0");
    cudaStream_t s = nullptr;
    EntryStream es(s);
    CKS(alloc_fix_state(h));
    DevBuf<float> gd;
    CK(gd.alloc(h->G.n));
    CKS(upload_field(h, g, h->G.n, gd.p, h->nM.p + 2, s, "g"));
    msc_status st = h->D == 3 ? verify_impl<3>(h, gd.p, xi, s, out) : verify_impl<2>(h, gd.p, xi, s, out);
    prof_flush(h);
    return st;
}

void msc_free_edits(msc_edits *e)
{
    if (!e) return;
    host_give(e->q_map);
    host_give(e->lossless_idx);
    host_give(e->lossless_val);
    free(e->trace);
    memset(e, 0, sizeof *e);
}

void msc_destroy(msc_handle *h)
{
    if (!h) return;
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    EntryStream es(nullptr);
    delete h;   // DevBuf members free their device memory
}

msc_status msc_fix_batch(msc_handle **hs, const float **f_hats, const float *xis, int n, const msc_options *opt,
                         msc_edits *outs, float **g_outs)
{
    g_last_error.clear();
    if (n < 0 || (n > 0 && (!hs || !f_hats || !xis || !outs || !g_outs))) return fail(MSC_ERR_INVALID_ARG, "bad batch arguments");
    for (int i = 0; i < n; i++) {
        if (!hs[i]) return fail(MSC_ERR_INVALID_ARG, "job %d has no handle", i);
        for (int j = 0; j < i; j++)
            if (hs[j] == hs[i]) return fail(MSC_ERR_INVALID_ARG, "jobs %d and %d share a handle", j, i);
    }
    if (n == 0) return MSC_OK;
    msc_options o;
    if (opt) o = *opt; else fill_defaults(&o);
    CKS(check_options(&o));
    CKS(device_ready());
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // the jobs start after the work already queued on the caller's stream (their inputs)
    cudaEvent_t ready = nullptr;
    CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CK(cudaEventRecord(ready, (cudaStream_t)o.stream));
    sm_count();
    std::vector<msc_status> st((size_t)n, MSC_OK);
    std::vector<std::string> msg((size_t)n);
    std::atomic<int> next{0};
    auto worker = [&]() {
        cudaStream_t ws = nullptr;
        cudaError_t e = cudaSetDevice(dev);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ws, ready, 0);
        for (int i; (i = next.fetch_add(1)) < n;) {
            if (e != cudaSuccess) {
                st[(size_t)i] = MSC_ERR_CUDA;
                msg[(size_t)i] = cudaGetErrorString(e);
                continue;
            }
            msc_options oi = o;
            oi.stream = ws;
            msc_rt::share_device(hs[i], std::min(n, BATCH_STREAMS));
            st[(size_t)i] = msc_fix(hs[i], f_hats[i], xis[i], &oi, outs + i, g_outs[i]);
            if (st[(size_t)i] != MSC_OK) msg[(size_t)i] = g_last_error;
        }
        if (ws) cudaStreamDestroy(ws);
    };
    const int nw = std::min(n, BATCH_STREAMS);
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; w++) pool.emplace_back(worker);
    for (auto &t : pool) t.join();
    cudaEventDestroy(ready);
    for (int i = 0; i < n; i++)
        if (st[(size_t)i] != MSC_OK) return fail(st[(size_t)i], "batch job %d: %s", i, msg[(size_t)i].c_str());
    return MSC_OK;
}

uint64_t msc_packed_bytes(uint64_t n_vertices, uint64_t n_lossless, int q_max)
{
    if (q_max < 1 || q_max > 7) return 0;
    return packed_size(n_vertices, n_lossless, q_max);
}

msc_status msc_pack_edits(const msc_edits *e, int q_max, uint8_t *out, uint64_t cap, uint64_t *n_out)
{
    g_last_error.clear();
    if (!e || !n_out) return fail(MSC_ERR_INVALID_ARG, "edits and n_out must be non-NULL");
    if (q_max < 1 || q_max > 7) return fail(MSC_ERR_INVALID_ARG, "q_max must be in 1..7");
    const uint64_t n = e->n_vertices, nl = e->n_lossless;
    if (n == 0 || n >= (1ull << 31) || !e->q_map) return fail(MSC_ERR_INVALID_ARG, "edits hold no q-map");
    if (nl && (!e->lossless_idx || !e->lossless_val)) return fail(MSC_ERR_INVALID_ARG, "edits lack their lossless values");
    const int b = pack_bits(q_max);
    const uint64_t size = packed_size(n, nl, q_max), nbits = ((n + 7) / 8) * b;
    *n_out = size;
    if (!out && cap == 0) return MSC_OK;   // size query
    if (!out || cap < size) return fail(MSC_ERR_INVALID_ARG, "output buffer holds %llu bytes, the record needs %llu",
                                        (unsigned long long)cap, (unsigned long long)size);
    CKS(device_ready());
    cudaStream_t s = nullptr;
    EntryStream es(s);
    DevBuf<uint8_t> qm, bits;
    DevBuf<uint64_t> idx, given;
    CK(qm.alloc(n));
    CK(cudaMemcpyAsync(qm.p, e->q_map, n, copy_kind(qm.p, e->q_map), s));
    uint64_t cnt = 0, nq = 0;
    CKS(lossless_positions(qm.p, n, q_max, idx, &cnt, &nq, s));
    if (cnt != nl) return fail(MSC_ERR_INVALID_ARG, "q-map marks %llu lossless vertices, edits list %llu",
                               (unsigned long long)cnt, (unsigned long long)nl);
    if (nl) {
        DevBuf<unsigned long long> bad;
        CK(bad.alloc(1));
        CK(cudaMemsetAsync(bad.p, 0, 8, s));
        CK(given.alloc(nl));
        CK(cudaMemcpyAsync(given.p, e->lossless_idx, nl * 8, copy_kind(given.p, e->lossless_idx), s));
        k_count_diff<<<grid_occ((const void *)k_count_diff, nl), TPB, 0, s>>>(idx.p, given.p, nl, bad.p);
        CK(cudaGetLastError());
        unsigned long long nbad = 0;
        CK(cudaMemcpyAsync(&nbad, bad.p, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (nbad) return fail(MSC_ERR_INVALID_ARG, "lossless_idx does not list the lossless vertices in increasing order");
    }
    CK(bits.alloc(nbits));
    k_pack_q<<<grid_occ((const void *)k_pack_q, (n + 7) / 8), TPB, 0, s>>>(qm.p, n, b, bits.p);
    CK(cudaGetLastError());
    uint8_t head[32] = {'M', 'S', 'C', 'E', 1, (uint8_t)q_max, (uint8_t)b, 0};
    put_u64(head + 8, n);
    put_u64(head + 16, nl);
    CK(cudaMemcpyAsync(out, head, 32, copy_kind(out, head), s));
    CK(cudaMemcpyAsync(out + 32, bits.p, nbits, copy_kind(out + 32, bits.p), s));
    if (nl) CK(cudaMemcpyAsync(out + 32 + nbits, e->lossless_val, nl * 4, copy_kind(out + 32 + nbits, e->lossless_val), s));
    CK(cudaStreamSynchronize(s));
    return MSC_OK;
}

msc_status msc_unpack_edits(const uint8_t *buf, uint64_t size, msc_edits *out, int *q_max)
{
    g_last_error.clear();
    if (!buf || !out || !q_max) return fail(MSC_ERR_INVALID_ARG, "buf, out and q_max must be non-NULL");
    memset(out, 0, sizeof *out);
    if (size < 32) return fail(MSC_ERR_INVALID_ARG, "not a packed edit record (%llu bytes)", (unsigned long long)size);
    CKS(device_ready());
    cudaStream_t s = nullptr;
    EntryStream es(s);
    uint8_t head[32];
    CK(cudaMemcpyAsync(head, buf, 32, copy_kind(head, buf), s));
    CK(cudaStreamSynchronize(s));
    const int qm_max = head[5], b = head[6];
    const uint64_t n = get_u64(head + 8), nl = get_u64(head + 16);
    if (memcmp(head, "MSCE", 4) != 0 || head[4] != 1 || qm_max < 1 || qm_max > 7 || b != pack_bits(qm_max))
        return fail(MSC_ERR_INVALID_ARG, "not a packed edit record (bad header)");
    if (n == 0 || n >= (1ull << 31) || nl > n || packed_size(n, nl, qm_max) != size)
        return fail(MSC_ERR_INVALID_ARG, "packed edit record of %llu bytes does not match its header", (unsigned long long)size);
    const uint64_t nbits = ((n + 7) / 8) * b;
    DevBuf<uint8_t> bits, qm;
    DevBuf<uint64_t> idx;
    DevBuf<unsigned long long> bad;
    CK(bits.alloc(nbits));
    CK(qm.alloc(n));
    CK(bad.alloc(1));
    CK(cudaMemcpyAsync(bits.p, buf + 32, nbits, copy_kind(bits.p, buf + 32), s));
    CK(cudaMemsetAsync(bad.p, 0, 8, s));
    k_unpack_q<<<grid_occ((const void *)k_unpack_q, (n + 7) / 8), TPB, 0, s>>>(bits.p, n, b, qm_max, qm.p, bad.p);
    CK(cudaGetLastError());
    unsigned long long nbad = 0;
    CK(cudaMemcpyAsync(&nbad, bad.p, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nbad) return fail(MSC_ERR_INVALID_ARG, "packed q-map holds %llu codes above q_max", nbad);
    uint64_t cnt = 0, nq = 0;
    CKS(lossless_positions(qm.p, n, qm_max, idx, &cnt, &nq, s));
    if (cnt != nl) return fail(MSC_ERR_INVALID_ARG, "packed q-map marks %llu lossless vertices, header says %llu",
                               (unsigned long long)cnt, (unsigned long long)nl);
    out->q_map = (uint8_t *)host_take(n);
    out->lossless_idx = (uint64_t *)host_take(nl ? nl * 8 : 8);
    out->lossless_val = (float *)host_take(nl ? nl * 4 : 4);
    if (!out->q_map || !out->lossless_idx || !out->lossless_val) {
        msc_free_edits(out);
        return fail(MSC_ERR_OOM, "host allocation of edits failed");
    }
    CK(cudaMemcpyAsync(out->q_map, qm.p, n, cudaMemcpyDeviceToHost, s));
    if (nl) {
        CK(cudaMemcpyAsync(out->lossless_idx, idx.p, nl * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(out->lossless_val, buf + 32 + nbits, nl * 4, copy_kind(out->lossless_val, buf + 32 + nbits), s));
    }
    CK(cudaStreamSynchronize(s));
    out->n_vertices = n;
    out->n_lossless = nl;
    out->n_quant = nq;
    *q_max = qm_max;
    return MSC_OK;
}

msc_status msc_tile_report(int nx, int ny, int nz, int *chosen, int *shapes, float *ms, int cap, int *n)
{
    g_last_error.clear();
    if (!n) return fail(MSC_ERR_INVALID_ARG, "n is NULL");
    *n = N_TILE_SHAPES;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
    TileTuning tt;
    bool tuned = false;
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        auto it = g_tile_tuned.find(std::make_tuple(dev, nx, ny, nz));
        if (it != g_tile_tuned.end()) { tt = it->second; tuned = true; }
    }
    for (int i = 0; i < N_TILE_SHAPES && i < cap; i++) {
        if (shapes) { shapes[3 * i] = 32; shapes[3 * i + 1] = TILE_SHAPES[i].ty; shapes[3 * i + 2] = TILE_SHAPES[i].zs; }
        if (ms) ms[i] = tuned ? tt.ms[i] : 0.f;
    }
    if (chosen) {
        chosen[0] = tuned ? 32 : 0;
        chosen[1] = tuned ? TILE_SHAPES[tt.best].ty : 0;
        chosen[2] = tuned ? TILE_SHAPES[tt.best].zs : 0;
    }
    return MSC_OK;
}

uint64_t msc_kv_bytes(uint64_t n_pairs) { return 32 + 8 * n_pairs; }

msc_status msc_pack_edits_kv(const msc_edits *e, uint8_t *out, uint64_t cap, uint64_t *n_out)
{
    g_last_error.clear();
    if (!e || !n_out) return fail(MSC_ERR_INVALID_ARG, "edits and n_out must be non-NULL");
    if (e->n_quant) return fail(MSC_ERR_INVALID_ARG, "%llu quantised counts: only floating edits (every edited vertex "
                                "stored as a value) form key-value pairs", (unsigned long long)e->n_quant);
    if (e->n_vertices == 0 || e->n_vertices >= (1ull << 31) || e->n_lossless > e->n_vertices)
        return fail(MSC_ERR_INVALID_ARG, "bad edit record sizes");
    if (e->n_lossless && (!e->lossless_idx || !e->lossless_val)) return fail(MSC_ERR_INVALID_ARG, "edits lack their pairs");
    const uint64_t nl = e->n_lossless, size = msc_kv_bytes(nl);
    *n_out = size;
    if (!out && cap == 0) return MSC_OK;
    if (!out || cap < size) return fail(MSC_ERR_INVALID_ARG, "out holds %llu bytes, the record needs %llu",
                                        (unsigned long long)cap, (unsigned long long)size);
    uint8_t head[32] = {'M', 'S', 'C', 'E', 2, 0, 0, 0};
    put_u64(head + 8, e->n_vertices);
    put_u64(head + 16, nl);
    memcpy(out, head, 32);
    uint8_t *ip = out + 32, *vp = out + 32 + 4 * nl;
    for (uint64_t k = 0; k < nl; k++) {
        const uint64_t v = e->lossless_idx[k];
        if (v >= e->n_vertices || (k && v <= e->lossless_idx[k - 1]))
            return fail(MSC_ERR_INVALID_ARG, "lossless_idx must be increasing vertex ids");
        for (int b = 0; b < 4; b++) ip[4 * k + b] = (uint8_t)(v >> (8 * b));
    }
    memcpy(vp, e->lossless_val, 4 * nl);
    return MSC_OK;
}

msc_status msc_unpack_edits_kv(const uint8_t *buf, uint64_t size, msc_edits *out)
{
    g_last_error.clear();
    if (!buf || !out) return fail(MSC_ERR_INVALID_ARG, "buf and out must be non-NULL");
    memset(out, 0, sizeof *out);
    if (size < 32 || memcmp(buf, "MSCE", 4) != 0 || buf[4] != 2) return fail(MSC_ERR_INVALID_ARG, "not a key-value edit record");
    const uint64_t n = get_u64(buf + 8), nl = get_u64(buf + 16);
    if (n == 0 || n >= (1ull << 31) || nl > n || msc_kv_bytes(nl) != size)
        return fail(MSC_ERR_INVALID_ARG, "key-value record of %llu bytes does not match its header", (unsigned long long)size);
    out->q_map = (uint8_t *)host_take(n);
    out->lossless_idx = (uint64_t *)host_take(nl ? nl * 8 : 8);
    out->lossless_val = (float *)host_take(nl ? nl * 4 : 4);
    if (!out->q_map || !out->lossless_idx || !out->lossless_val) {
        msc_free_edits(out);
        return fail(MSC_ERR_OOM, "host allocation of edits failed");
    }
    memset(out->q_map, 0, n);
    const uint8_t *ip = buf + 32;
    for (uint64_t k = 0; k < nl; k++) {
        uint64_t v = 0;
        for (int b = 0; b < 4; b++) v |= (uint64_t)ip[4 * k + b] << (8 * b);
        if (v >= n || (k && v <= out->lossless_idx[k - 1])) {
            msc_free_edits(out);
            return fail(MSC_ERR_INVALID_ARG, "key-value record holds an out-of-order or out-of-range vertex");
        }
        out->lossless_idx[k] = v;
        out->q_map[v] = MSC_QMAP_LOSSLESS;
    }
    memcpy(out->lossless_val, buf + 32 + 4 * nl, 4 * nl);
    out->n_vertices = n;
    out->n_lossless = nl;
    return MSC_OK;
}

msc_status msc_critical_cells_static(const float *field, int nx, int ny, int nz, int64_t *rows, int32_t *dims,
                                     uint64_t cap, uint64_t *n_out, void *stream)
{
    g_last_error.clear();
    if (!field || !n_out) return fail(MSC_ERR_INVALID_ARG, "field and n_out must be non-NULL");
    CKS(check_dims(nx, ny, nz));
    const unsigned long long n = (unsigned long long)nx * ny * nz;
    if (n > MSC_STATIC_MAX_VERTICES)
        return fail(MSC_ERR_INVALID_ARG, "grid of %llu vertices exceeds the static scratch limit of %u vertices", n,
                    (unsigned)MSC_STATIC_MAX_VERTICES);
    if (cap && (!rows || !dims)) return fail(MSC_ERR_INVALID_ARG, "rows and dims must be non-NULL when cap > 0");
    CKS(device_ready());
    if (!on_current_device(field) || (cap && (!on_current_device(rows) || !on_current_device(dims))))
        return fail(MSC_ERR_INVALID_ARG, "field, rows and dims must be device pointers on the current device");
    const Grid G = make_grid(nx, ny, nz);
    cudaStream_t s = (cudaStream_t)stream;
    return nz > 1 ? critical_static<3>(field, G, rows, dims, cap, n_out, s)
                  : critical_static<2>(field, G, rows, dims, cap, n_out, s);
}

msc_status msc_selftest_barrier(int timeout_ms, void *stream)
{
    g_last_error.clear();
    if (timeout_ms < 1 || timeout_ms > 2000) return fail(MSC_ERR_INVALID_ARG, "timeout_ms must be 1..2000");
    CKS(device_ready());
    cudaStream_t s = (cudaStream_t)stream;
    EntryStream es(s);
    DevBuf<GridBarrier> gb;
    DevBuf<LoopState> ls;
    CK(gb.alloc(1));
    CK(ls.alloc(1));
    CK(cudaMemsetAsync(gb.p, 0, sizeof(GridBarrier), s));
    CK(cudaMemsetAsync(ls.p, 0, sizeof(LoopState), s));
    k_barrier_selftest<<<2, 32, 0, s>>>(gb.p, ls.p, (unsigned long long)timeout_ms * 1000000ull);
    CK(cudaGetLastError());
    LoopState L{};
    CK(cudaMemcpyAsync(&L, ls.p, sizeof L, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (L.status == MSC_ERR_DEVICE_TIMEOUT && L.halt)
        return fail(MSC_ERR_DEVICE_TIMEOUT, "the barrier wait gave up as it should");
    return fail(MSC_ERR_CUDA, "the barrier wait did not report its timeout (status %d)", L.status);
}

msc_status msc_release_cached_memory(void)
{
    g_last_error.clear();
    CKS(device_ready());
    CK(cudaDeviceSynchronize());
    host_trim();
    cudaMemPool_t pool = lib_pool();
    if (pool) CK(cudaMemPoolTrimTo(pool, 0));
    return MSC_OK;
}

msc_status msc_set_walk_limits(uint32_t warp_stack, uint32_t local_steps)
{
    g_last_error.clear();
    if (warp_stack > (uint32_t)SS_WARP_STACK)
        return fail(MSC_ERR_INVALID_ARG, "warp_stack must be at most %d", SS_WARP_STACK);
    g_walk_stack.store(warp_stack ? warp_stack : (uint32_t)SS_WARP_STACK);
    g_walk_steps.store(local_steps ? local_steps : TRI_LOCAL_STEPS);
    return MSC_OK;
}

uint64_t msc_inject_alloc_failures(uint64_t after, uint64_t count)
{
    g_inject_left.store(0);
    g_inject_after.store(after);
    g_inject_left.store(count);
    return g_injected.load();
}

msc_status msc_pool_used_bytes(uint64_t *used)
{
    g_last_error.clear();
    if (!used) return fail(MSC_ERR_INVALID_ARG, "used is NULL");
    *used = 0;
    CKS(device_ready());
    cudaMemPool_t pool = lib_pool();
    if (!pool) return fail(MSC_ERR_CUDA, "the library's memory pool could not be created");
    uint64_t v = 0;
    CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
    *used = (uint64_t)v;
    return MSC_OK;
}

msc_status msc_get_stats(msc_handle *h, msc_stats *out)
{
    if (!h || !out) return fail(MSC_ERR_INVALID_ARG, "handle and out must be non-NULL");
    memset(out, 0, sizeof *out);
    for (int i = 0; i < 12; i++) {
        out->launches[i] = h->launches[i];
        out->ms[i] = h->ms[i];
        out->timed_launches[i] = h->timed[i];
        out->items[i] = h->items[i];
    }
    for (int i = 0; i < 3; i++) out->round_work[i] = h->round_work[i];
    for (int i = 0; i < 4; i++) out->round_phase_ms[i] = h->round_phase_ns[i] * 1e-6;
    out->cluster_launches = h->cluster_launches;
    out->cluster_rounds = h->cluster_rounds;
    return MSC_OK;
}

msc_status msc_reset_stats(msc_handle *h)
{
    if (!h) return fail(MSC_ERR_INVALID_ARG, "handle is NULL");
    for (int i = 0; i < 12; i++) { h->launches[i] = 0; h->ms[i] = 0.0; h->timed[i] = 0; h->items[i] = 0; }
    for (int i = 0; i < 3; i++) h->round_work[i] = 0;
    for (int i = 0; i < 4; i++) h->round_phase_ns[i] = 0;
    h->cluster_launches = h->cluster_rounds = 0;
    return MSC_OK;
}

msc_status msc_gradient_pairs(const float *field, int nx, int ny, int nz, int64_t *rows, uint64_t cap, uint64_t *n_out)
{
    g_last_error.clear();
    if (!n_out) return fail(MSC_ERR_INVALID_ARG, "n_out is NULL");
    CKS(check_dims(nx, ny, nz));
    CKS(device_ready());
    const Grid G = make_grid(nx, ny, nz);
    return nz > 1 ? introspect<3>(field, G, 0, rows, nullptr, cap, n_out) : introspect<2>(field, G, 0, rows, nullptr, cap, n_out);
}

msc_status msc_critical_cells(const float *field, int nx, int ny, int nz, int64_t *rows, int32_t *dims, uint64_t cap,
                              uint64_t *n_out)
{
    g_last_error.clear();
    if (!n_out) return fail(MSC_ERR_INVALID_ARG, "n_out is NULL");
    CKS(check_dims(nx, ny, nz));
    CKS(device_ready());
    const Grid G = make_grid(nx, ny, nz);
    return nz > 1 ? introspect<3>(field, G, 1, rows, dims, cap, n_out) : introspect<2>(field, G, 1, rows, dims, cap, n_out);
}

}  // extern "C"
