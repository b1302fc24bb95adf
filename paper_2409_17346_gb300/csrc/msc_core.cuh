// Per-element logic of the fix loop: one anchor, one target vertex, one separatrix seed.
// The __global__ kernels in msc_lib.cu are thin grid-stride wrappers around these.
#pragma once
#include <cstdint>
#include "msc_cells.cuh"

namespace msc {

// tables read with run-time indices (the dense evaluator uses compile-time copies)
#ifdef __CUDACC__
static __device__ const Tab<2> kTab2 = make_tab<2>();
static __device__ const Tab<3> kTab3 = make_tab<3>();
#endif
#ifdef MSC_HOST_EMULATION
static const Tab<2> hTab2 = make_tab<2>();
static const Tab<3> hTab3 = make_tab<3>();
#endif
template <int D> MSC_HD inline const Tab<D> &rt_tab();
template <> MSC_HD inline const Tab<2> &rt_tab<2>()
{
#if defined(__CUDA_ARCH__) || !defined(MSC_HOST_EMULATION)
    return kTab2;
#else
    return hTab2;
#endif
}
template <> MSC_HD inline const Tab<3> &rt_tab<3>()
{
#if defined(__CUDA_ARCH__) || !defined(MSC_HOST_EMULATION)
    return kTab3;
#else
    return hTab3;
#endif
}

// The tables of the 3D walks, one word per cell type, so that a lookup with a type that
// differs from lane to lane is one load rather than one per field:
//  nb[n]: neighbour offset n of a vertex, bits 0-1, 2-3, 4-5: x, y, z plus one;
//  asc[t][j]: ascending step of a tet of type t whose lowest corner is slot j (asc_off,
//    asc_type), bits 0-1, 2-3, 4-5: x, y, z offsets plus one, bits 8-10: the next tet's type;
//  tri[t], byte j (j < 3): facet edge j of a triangle of type t, bits 0-2 its anchor offset
//    (x, y, z, each 0 or 1), bits 3-5 its edge type; bits 24-29: tri_opp[t][0..2], 2 bits each;
//  ecof[e], byte i (i < 6): cofacet triangle i of an edge of type e, bits 0-2 minus its anchor
//    offset (each offset is 0 or -1), bits 4-7 its triangle type.
struct TriPack {
    uint32_t nb[14];
    uint32_t asc[6][4];
    uint32_t tri[12];
    uint64_t ecof[7];
};
constexpr TriPack make_tri_pack()
{
    constexpr Tab<3> T = make_tab<3>();
    TriPack k{};
    for (int n = 0; n < 14; n++)
        k.nb[n] = (uint32_t)(T.nb[n][0] + 1) | (uint32_t)(T.nb[n][1] + 1) << 2 | (uint32_t)(T.nb[n][2] + 1) << 4;
    for (int t = 0; t < 6; t++)
        for (int j = 0; j < 4; j++)
            k.asc[t][j] = (uint32_t)(T.asc_off[t][j][0] + 1) | (uint32_t)(T.asc_off[t][j][1] + 1) << 2 |
                          (uint32_t)(T.asc_off[t][j][2] + 1) << 4 | (uint32_t)T.asc_type[t][j] << 8;
    for (int t = 0; t < 12; t++) {
        uint32_t w = 0;
        for (int j = 0; j < 3; j++) {
            const uint32_t b = (uint32_t)T.tfac_anc[t][j][0] | (uint32_t)T.tfac_anc[t][j][1] << 1 |
                               (uint32_t)T.tfac_anc[t][j][2] << 2 | (uint32_t)T.tfac_type[t][j] << 3;
            w |= b << (8 * j);
            w |= (uint32_t)T.tri_opp[t][j] << (24 + 2 * j);
        }
        k.tri[t] = w;
    }
    for (int e = 0; e < 7; e++) {
        uint64_t w = 0;
        for (int i = 0; i < T.necof[e]; i++) {
            const uint64_t b = (uint64_t)-T.ecof_anc[e][i][0] | (uint64_t)-T.ecof_anc[e][i][1] << 1 |
                               (uint64_t)-T.ecof_anc[e][i][2] << 2 | (uint64_t)T.ecof_type[e][i] << 4;
            w |= b << (8 * i);
        }
        k.ecof[e] = w;
    }
    return k;
}
#ifdef __CUDACC__
static __device__ const TriPack kTriPack = make_tri_pack();
#endif
#ifdef MSC_HOST_EMULATION
static const TriPack hTriPack = make_tri_pack();
#endif
MSC_HD inline const TriPack &rt_tri_pack()
{
#if defined(__CUDA_ARCH__) || !defined(MSC_HOST_EMULATION)
    return kTriPack;
#else
    return hTriPack;
#endif
}

// For a ring offset r (a vertex u = v + r whose order against an edited vertex v may flip):
// bit i set iff the anchor p = v - win[i] (whose window holds v) also holds u in its window.
// An anchor's code compares only vertices of its window, so a flip of (v, u) can change only
// those anchors, and the anchors to refresh are the union over the flipped pairs.
template <int D> struct RingWin {
    uint64_t m[64];
};
template <int D> constexpr RingWin<D> make_ring_win()
{
    constexpr Tab<D> T = make_tab<D>();
    RingWin<D> rw{};
    for (int j = 0; j < T.nring; j++)
        for (int i = 0; i < T.nwin; i++) {
            const int o[3] = {T.win[i][0] + T.ring[j][0], T.win[i][1] + T.ring[j][1], T.win[i][2] + T.ring[j][2]};
            bool in = false;
            for (int k = 0; k < T.nwin; k++)
                if (T.win[k][0] == o[0] && T.win[k][1] == o[1] && T.win[k][2] == o[2]) in = true;
            if (in) rw.m[j] |= 1ull << i;
        }
    return rw;
}
static_assert(make_tab<3>().nwin <= 64 && make_tab<3>().nring <= 64, "masks hold 64 positions");
#ifdef __CUDACC__
static __device__ const RingWin<2> kRingWin2 = make_ring_win<2>();
static __device__ const RingWin<3> kRingWin3 = make_ring_win<3>();
#endif
#ifdef MSC_HOST_EMULATION
static const RingWin<2> hRingWin2 = make_ring_win<2>();
static const RingWin<3> hRingWin3 = make_ring_win<3>();
#endif
template <int D> MSC_HD inline const RingWin<D> &rt_ring_win();
template <> MSC_HD inline const RingWin<2> &rt_ring_win<2>()
{
#if defined(__CUDA_ARCH__) || !defined(MSC_HOST_EMULATION)
    return kRingWin2;
#else
    return hRingWin2;
#endif
}
template <> MSC_HD inline const RingWin<3> &rt_ring_win<3>()
{
#if defined(__CUDA_ARCH__) || !defined(MSC_HOST_EMULATION)
    return kRingWin3;
#else
    return hRingWin3;
#endif
}

constexpr uint8_t ST_FLOOR = 0xF0;   // g == lb, stored losslessly (Eq. 2 "otherwise")
constexpr uint8_t ST_EXACT = 0xF1;   // g == f, stored losslessly (stuck-case restore)

struct Grid {
    int nx, ny, nz;
    uint32_t n;
    // reciprocals of nx and ny: v / d == (v * m) >> s for every v < 2^31 (make_grid)
    uint64_t mx, my;
    int sx, sy;
};

// Division by an invariant integer as a multiply and a shift (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994, Thm 4.2): for 31-bit
// dividends and 2^(l-1) < d <= 2^l, m = ceil(2^(31+l) / d) gives floor(v / d) =
// floor(v * m / 2^(31+l)); v * m < 2^63.
__host__ __device__ inline void div_magic(uint32_t d, uint64_t &m, int &s)
{
    int l = 0;
    while ((1ull << l) < d) l++;
    s = 31 + l;
    m = ((1ull << s) + d - 1) / d;
}

__host__ __device__ inline Grid make_grid(int nx, int ny, int nz)
{
    Grid G{};
    G.nx = nx; G.ny = ny; G.nz = nz;
    G.n = (uint32_t)((uint64_t)nx * ny * nz);
    div_magic((uint32_t)nx, G.mx, G.sx);
    div_magic((uint32_t)ny, G.my, G.sy);
    return G;
}

struct Counters {
    unsigned long long ncase, nlive, nT, nX, sumT, sumX;   // targeting pass
    unsigned long long nE, nD, nM, novf, err, nSD;
    unsigned long long steps[4];                           // cells stepped: desc, asc, saddle
    unsigned long long rep[16];                            // verify / misc
    unsigned long long wnext;                              // C-pass: next listed block to take
};

// device-side state of the edit loop, so rounds can run back to back without the host
struct LoopState {
    int halt;                 // the current phase is over (no false case left) or an error
    int status;               // 0 running / done, 4 max_iters reached, 6 stalled
    int track_dirty;          // accumulate dirty anchors for the separatrix state
    int leave;                // the round graph's remaining rounds do nothing: a round edited
                              // few vertices, and the persistent round kernel takes over
    unsigned iters, n_c, n_s, n_fb;
    unsigned max_iters, exact_fallback, trace_cap, ntrace;
    unsigned long long nSD;
    unsigned long long edit_items, refresh_items, cpass_items, cases;
    unsigned long long nblk;  // entries of the C-block list for the next C-pass
    unsigned long long last_items;   // vertices the last round edited (targets + restores)
    unsigned long long nbl[2];       // persistent round kernel: entries of its two C-block lists
    int rounds_kernel;               // small rounds run in the persistent round kernel
    int pad;
    unsigned long long small_round;  // a round that edits fewer vertices hands the next to it
    unsigned long long phase_ns[4];  // persistent round kernel: device time per phase (block 0's
                                     // view: from one barrier's exit to the next's)
};

// everything a kernel of one job needs (device pointers)
struct Ctx {
    Grid G;
    int tier, qmax, exact_fallback;
    int qcap;                        // quantised steps a vertex may take before the floor:
                                     // q_max (Eq. 2), or no cap in floating-edit mode
    float xi, step;
    const float *f, *fhat;
    float *g;
    float *gprev;                    // value before the current round, for vertices in T u X
    uint8_t *state;
    const uint64_t *code_f;
    const uint64_t *low_f;           // 3D: per anchor, the f-lowest vertex slot of each triangle
                                     // t (bits 2t) and tetrahedron k (bits 24 + 2k)
    uint64_t *code_g;
    uint32_t *Tbits, *Xbits, *Dbits;
    uint32_t *Tlist, *Xlist, *Dlist;
    uint32_t *Elist;                 // vertices whose value the current round changed
    uint32_t *vis_v, *vis_top, *vis_tri;
    uint32_t *ovf_in, *ovf_out;      // saddle-saddle spill queues: (triangle id, entry edge) pairs
    uint32_t ovf_cap;
    uint32_t ss_stack_cap;           // entries of a warp's saddle-saddle stack in use (<= its size)
    uint32_t tri_local_steps;        // steps one thread walks before it spills the rest
    Counters *cnt;
    // persistent separatrix state (tier 4): one byte per node, see "separatrix state" below
    uint32_t *ns_v, *ns_top, *ns_tri, *ns_dead;   // separatrix node words, two per uint32
    uint32_t *sDbits, *sDlist;       // anchors dirtied since the last S-pass
    LoopState *ls;
    uint32_t *Mbits;                 // anchors whose code differs from f's
    uint32_t *Cbits;                 // anchors whose critical cells differ from f's (tier restricted)
    uint32_t *Csum;                  // one bit per block of 32 Cbits words (1024 anchors): the
                                     // block may hold a set bit (cleared lazily when found empty)
    uint32_t *Cblk;                  // blocks whose Csum bit is set, listed for the next C-pass
    int64_t *trace;                  // rows (kind, |T|, |X|, sum T, sum X), ls->trace_cap rows
    unsigned long long *tally;       // when set: per-block (cases, live cases) in shared memory
    int mark_only;                   // add_case only sets the target's T bit (no return value
                                     // awaited); k_tlist lists the T bits afterwards
    float *fuse_g;                   // when set (persistent round kernel): the C-pass thread that
                                     // lists a new target edits it at once, writing fuse_g (the
                                     // live g) while the round's cases read g (here the pre-round
                                     // copy); the state follows in the mark phase
    // verification of saddle-saddle connectors: triangles from which the walk found a
    // troublemaker (bitset over triangle ids, plus a list of them, ss_cap entries)
    uint32_t *ss_bad, *ss_list;
    unsigned long long *ss_n;
    uint32_t ss_cap;
};

// ------------------------------------------------------------------------------------
// atomics and correctly rounded float operations
// ------------------------------------------------------------------------------------
#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned a_or(uint32_t *p, uint32_t v) { return atomicOr(p, v); }
__device__ __forceinline__ unsigned long long a_add(unsigned long long *p, unsigned long long v) { return atomicAdd(p, v); }
__device__ __forceinline__ uint32_t a_exch(uint32_t *p, uint32_t v) { return atomicExch(p, v); }
__device__ __forceinline__ float sub_ru(float a, float b) { return __fsub_ru(a, b); }
__device__ __forceinline__ float add_rd(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
template <class T> __device__ __forceinline__ T ld(const T *p) { return __ldg(p); }
#else
float emu_sub_ru(float a, float b);
float emu_add_rd(float a, float b);
inline unsigned a_or(uint32_t *p, uint32_t v) { unsigned o = *p; *p |= v; return o; }
inline unsigned long long a_add(unsigned long long *p, unsigned long long v) { unsigned long long o = *p; *p += v; return o; }
inline uint32_t a_exch(uint32_t *p, uint32_t v) { uint32_t o = *p; *p = v; return o; }
inline float sub_ru(float a, float b) { return emu_sub_ru(a, b); }
inline float add_rd(float a, float b) { return emu_add_rd(a, b); }
inline float sub_rn(float a, float b) { volatile float r = a - b; return r; }
inline float mul_rn(float a, float b) { volatile float r = a * b; return r; }
template <class T> inline T ld(const T *p) { return *p; }
#endif

// add v to a hot counter: one atomic per group of converged threads
#ifdef __CUDA_ARCH__
__device__ __forceinline__ void count_add(unsigned long long *p, unsigned long long v)
{
    const unsigned mask = __activemask();
    const unsigned lo = __reduce_add_sync(mask, (unsigned)(v & 0xffffffffu));
    const unsigned hi = __reduce_add_sync(mask, (unsigned)(v >> 32));
    if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) atomicAdd(p, ((unsigned long long)hi << 32) + lo);
}
#else
inline void count_add(unsigned long long *p, unsigned long long v) { *p += v; }
#endif

// a case into a shared (cases, live cases) tally: one pair of atomics per group of converged
// threads (the lanes of a warp would otherwise queue on the same two words)
#ifdef __CUDA_ARCH__
__device__ __forceinline__ void tally_add(unsigned long long *t, bool live)
{
    const unsigned mask = __activemask();
    const unsigned nl = (unsigned)__popc(__ballot_sync(mask, live));
    if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
        atomicAdd(t, (unsigned long long)__popc(mask));
        if (nl) atomicAdd(t + 1, (unsigned long long)nl);
    }
}
#else
inline void tally_add(unsigned long long *t, bool live) { t[0] += 1; t[1] += live ? 1 : 0; }
#endif

// slot in a list whose length lives in *n: one atomic per group of converged threads
#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned long long list_slot(unsigned long long *n)
{
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(n, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}
#else
inline unsigned long long list_slot(unsigned long long *n) { return (*n)++; }
#endif

MSC_HD inline bool test_and_set(uint32_t *bits, uint32_t i)
{
    const uint32_t m = 1u << (i & 31);
    return (a_or(bits + (i >> 5), m) & m) != 0;
}

MSC_HD inline bool sos_lt(float a, uint32_t ia, float b, uint32_t ib)
{
    return a < b || (a == b && ia < ib);
}

MSC_HD inline void coords(const Grid &G, uint32_t v, int &x, int &y, int &z)
{
    const uint32_t t = (uint32_t)(((uint64_t)v * G.mx) >> G.sx);    // v / nx
    const uint32_t u = (uint32_t)(((uint64_t)t * G.my) >> G.sy);    // t / ny
    x = (int)(v - t * (uint32_t)G.nx);
    y = (int)(t - u * (uint32_t)G.ny);
    z = (int)u;
}

MSC_HD inline bool inside(const Grid &G, int x, int y, int z)
{
    return x >= 0 && y >= 0 && z >= 0 && x < G.nx && y < G.ny && z < G.nz;
}

MSC_HD inline uint32_t vid(const Grid &G, int x, int y, int z)
{
    return (uint32_t)x + (uint32_t)G.nx * ((uint32_t)y + (uint32_t)G.ny * (uint32_t)z);
}

// bit k set <=> cube corner k of the anchor at (x,y,z) is in the domain
template <int D> MSC_HD inline unsigned corner_mask(const Grid &G, int x, int y, int z)
{
    const bool cx = x + 1 < G.nx, cy = y + 1 < G.ny, cz = D == 3 && z + 1 < G.nz;
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < Tab<D>::NC; k++) {
        const bool in = (!(k & 1) || cx) && (!(k & 2) || cy) && (!(k & 4) || cz);
        m |= (unsigned)in << k;
    }
    return m;
}

// a value load: through the read-only data path (NC, for arrays that no thread writes while
// the kernel runs), or a plain coherent load (arrays that other blocks of a persistent
// kernel write between its grid barriers)
template <bool NC> MSC_HD __forceinline__ float ldv(const float *p)
{
    if constexpr (NC) return ld(p);
    else return *p;
}

// the window of values around an anchor (+inf outside the domain)
template <int D, bool NC = true> MSC_HD inline void load_window(const float *v, const Grid &G, int x, int y, int z, float *w)
{
    const float INF = pos_inf();
    constexpr int ZL = D == 3 ? -1 : 0, ZH = D == 3 ? 2 : 0;
#pragma unroll
    for (int dz = ZL; dz <= ZH; dz++)
#pragma unroll
        for (int dy = -1; dy <= 2; dy++)
#pragma unroll
            for (int dx = -1; dx <= 2; dx++) {
                const int xx = x + dx, yy = y + dy, zz = z + dz;
                w[wpos<D>(dx, dy, dz)] = inside(G, xx, yy, zz) ? ldv<NC>(v + vid(G, xx, yy, zz)) : INF;
            }
}

// window of an anchor at least one vertex from the lower and two from the upper faces
template <int D, bool NC = true> MSC_HD inline void load_window_interior(const float *v, const Grid &G, uint32_t p, float *w)
{
    constexpr int ZL = D == 3 ? -1 : 0, ZH = D == 3 ? 2 : 0;
    const int sy = G.nx, sz = G.nx * G.ny;
#pragma unroll
    for (int dz = ZL; dz <= ZH; dz++)
#pragma unroll
        for (int dy = -1; dy <= 2; dy++)
#pragma unroll
            for (int dx = -1; dx <= 2; dx++) {
                const bool lowcube = dx <= 1 && dy <= 1 && dz <= 1;
                const bool highcube = dx >= 0 && dy >= 0 && dz >= 0;
                if (lowcube || highcube) w[wpos<D>(dx, dy, dz)] = ldv<NC>(v + (int64_t)p + dx + dy * sy + dz * sz);
            }
}

template <int D, bool NC = true> MSC_HD inline uint64_t anchor_code(const float *v, const Grid &G, uint32_t p)
{
    int x, y, z;
    coords(G, p, x, y, z);
    float w[Tab<D>::WS];
    const bool interior = x >= 1 && y >= 1 && x + 2 < G.nx && y + 2 < G.ny && (D == 2 || (z >= 1 && z + 2 < G.nz));
    if (interior) {
        load_window_interior<D, NC>(v, G, p, w);
        return eval_anchor<D>(w, (1u << Tab<D>::NC) - 1u);
    }
    load_window<D, NC>(v, G, x, y, z, w);
    return eval_anchor<D>(w, corner_mask<D>(G, x, y, z));
}

// ------------------------------------------------------------------------------------
// small cell helpers (relative offsets -> absolute vertices)
// ------------------------------------------------------------------------------------
struct Verts {
    int n;
    uint32_t id[4];
    int x[4], y[4], z[4];
};

MSC_HD inline void vpush(Verts &V, const Grid &G, int x, int y, int z)
{
    V.x[V.n] = x; V.y[V.n] = y; V.z[V.n] = z;
    V.id[V.n] = vid(G, x, y, z);
    V.n++;
}

// anchored cell vertices: kind 0 vertex, 1 edge, 2 triangle, 3 tet
template <int D> MSC_HD inline Verts cell_verts(const Grid &G, int x, int y, int z, int kind, int t)
{
    const Tab<D> &T = rt_tab<D>();
    Verts V;
    V.n = 0;
    vpush(V, G, x, y, z);
    int cs[3] = {0, 0, 0}, nc = 0;
    if (kind == 1) { cs[0] = t + 1; nc = 1; }
    if (kind == 2) { cs[0] = T.tA[t]; cs[1] = T.tB[t]; nc = 2; }
    if (kind == 3) { cs[0] = T.kA[t]; cs[1] = T.kB[t]; cs[2] = 7; nc = 3; }
    for (int i = 0; i < nc; i++) vpush(V, G, x + (cs[i] & 1), y + ((cs[i] >> 1) & 1), z + ((cs[i] >> 2) & 1));
    return V;
}

template <bool NC = true> MSC_HD inline int lowest_of(const Verts &V, const float *vals)
{
    int lo = 0;
    float lv = ldv<NC>(vals + V.id[0]);
    for (int i = 1; i < V.n; i++) {
        const float vi = ldv<NC>(vals + V.id[i]);
        if (sos_lt(vi, V.id[i], lv, V.id[lo])) { lo = i; lv = vi; }
    }
    return lo;
}

// a false case: vertex t is lowered this round; a stuck case restores the closed 1-rings of
// the case cell's vertices to f (exact fallback)
MSC_HD inline void fuse_target(const Ctx &c, uint32_t t);

template <int D> MSC_HD inline void add_case(const Ctx &c, uint32_t t, const Verts &cell)
{
    const Tab<D> &T = rt_tab<D>();
    const uint8_t st = c.state[t];
    const bool live = st != ST_FLOOR && st != ST_EXACT;
    if (c.tally) {
        tally_add(c.tally, live);
    } else {
        count_add(&c.cnt->ncase, 1ull);
        if (live) count_add(&c.cnt->nlive, 1ull);
    }
    if (c.mark_only) {
#ifdef __CUDA_ARCH__
        atomicOr(c.Tbits + (t >> 5), 1u << (t & 31));
#else
        a_or(c.Tbits + (t >> 5), 1u << (t & 31));
#endif
    } else if (!test_and_set(c.Tbits, t)) {
        c.Tlist[list_slot(&c.cnt->nT)] = t;
        count_add(&c.cnt->sumT, (unsigned long long)t);
        if (c.fuse_g) fuse_target(c, t);
    }
    if (live || !c.exact_fallback) return;
    for (int i = 0; i < cell.n; i++) {
        for (int n = -1; n < T.NNB; n++) {
            int xx = cell.x[i], yy = cell.y[i], zz = cell.z[i];
            if (n >= 0) { xx += T.nb[n][0]; yy += T.nb[n][1]; zz += T.nb[n][2]; }
            if (!inside(c.G, xx, yy, zz)) continue;
            const uint32_t u = vid(c.G, xx, yy, zz);
            if (!test_and_set(c.Xbits, u)) {
                c.Xlist[list_slot(&c.cnt->nX)] = u;
                count_add(&c.cnt->sumX, (unsigned long long)u);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// C-pass (Sec. 4.3): false critical cells owned by one anchor
// ------------------------------------------------------------------------------------
MSC_HD inline bool crit_v(int f) { return f == 15; }
MSC_HD inline bool crit_c(int f) { return f == 0; }

// target of a false negative cell paired DOWN in g: its g-lowest vertex y; when y is also
// its f-lowest vertex, repair the f-pairing of the facet L = cell - y instead
template <int D>
MSC_HD inline uint32_t fn_down_target(const Ctx &c, int x, int y, int z, int kind, int t, const Verts &V)
{
    const Tab<D> &T = rt_tab<D>();
    const int jg = lowest_of<false>(V, c.g), jf = lowest_of(V, c.f);   // g: plain load (written by edits)
    if (jg != jf) return V.id[jf];
    if (kind == 1) {                       // L = the other vertex h
        const int h = 1 - jg;
        const int vf = vfield<D>(ld(c.code_f + V.id[h]));
        if (vf == 15) return V.id[h];
        return vid(c.G, V.x[h] + T.nb[vf][0], V.y[h] + T.nb[vf][1], V.z[h] + T.nb[vf][2]);
    }
    // facet opposite corner jg
    int ax, ay, az, ty;
    if (kind == 2) {
        const int corner = jg == 0 ? 0 : (jg == 1 ? T.tA[t] : T.tB[t]);
        int j = 0;
        for (int q = 0; q < 3; q++) if (T.tfac_opp[t][q] == corner) j = q;
        ax = x + T.tfac_anc[t][j][0]; ay = y + T.tfac_anc[t][j][1]; az = z + T.tfac_anc[t][j][2];
        ty = T.tfac_type[t][j];
        const uint32_t a = vid(c.G, ax, ay, az);
        const int ef = efield<D>(ld(c.code_f + a), ty);
        if (ef >= 2)
            return vid(c.G, ax + T.ecof_v[ty][ef - 2][0], ay + T.ecof_v[ty][ef - 2][1], az + T.ecof_v[ty][ef - 2][2]);
        Verts L = cell_verts<D>(c.G, ax, ay, az, 1, ty);
        return L.id[lowest_of(L, c.f)];
    }
    const int corner = jg == 0 ? 0 : (jg == 1 ? T.kA[t] : (jg == 2 ? T.kB[t] : 7));
    int j = 0;
    for (int q = 0; q < 4; q++) if (T.kfac_opp[t][q] == corner) j = q;
    ax = x + T.kfac_anc[t][j][0]; ay = y + T.kfac_anc[t][j][1]; az = z + T.kfac_anc[t][j][2];
    ty = T.kfac_type[t][j];
    const uint32_t a = vid(c.G, ax, ay, az);
    const int tf = tfield<D>(ld(c.code_f + a), ty);
    if (tf >= 2)
        return vid(c.G, ax + T.tcof_v[ty][tf - 2][0], ay + T.tcof_v[ty][tf - 2][1], az + T.tcof_v[ty][tf - 2][2]);
    Verts L = cell_verts<D>(c.G, ax, ay, az, 2, ty);
    return L.id[lowest_of(L, c.f)];
}

// Cells an anchor owns, numbered for the C-pass: 0 the vertex, 1 + e the edges,
// 1 + NE + t the triangles, 1 + NE + NT + k the tetrahedra.
// case_mask: bit i set iff cell i exists and is critical in exactly one of f and g (the
// tier's cells: tier 1 in 3D skips edges and triangles, tier 1 in 2D skips edges).
template <int D> MSC_HD inline uint32_t case_mask(const Ctx &c, uint32_t p, uint64_t cf, uint64_t cg)
{
    const Tab<D> &T = rt_tab<D>();
    if (cf == cg) return 0;
    int x, y, z;
    coords(c.G, p, x, y, z);
    const unsigned cin = corner_mask<D>(c.G, x, y, z);
    uint32_t m = crit_v(vfield<D>(cf)) != crit_v(vfield<D>(cg)) ? 1u : 0u;
    if (c.tier >= 2)
        for (int e = 0; e < T.NE; e++)
            if (((cin >> (e + 1)) & 1u) && crit_c(efield<D>(cf, e)) != crit_c(efield<D>(cg, e))) m |= 1u << (1 + e);
    if (D == 2 || c.tier >= 2)
        for (int tt = 0; tt < T.NT; tt++)
            if (((cin >> T.tB[tt]) & 1u) && crit_c(tfield<D>(cf, tt)) != crit_c(tfield<D>(cg, tt)))
                m |= 1u << (1 + T.NE + tt);
    if ((cin >> 7) & 1u)
        for (int k = 0; k < T.NK; k++)
            if (crit_c(kfield<D>(cf, k)) != crit_c(kfield<D>(cg, k))) m |= 1u << (1 + T.NE + T.NT + k);
    return m;
}

// the false case of cell i of anchor p (a bit of case_mask): false positive (critical in g
// only): lower the extra vertex of its f-partner; false negative (critical in f only): lower
// the cell's f-lowest vertex, or repair a facet (fn_down_target)
template <int D> MSC_HD inline void case_apply(const Ctx &c, uint32_t p, int i)
{
    const Tab<D> &T = rt_tab<D>();
    const uint64_t cf = ld(c.code_f + p), cg = c.code_g[p];
    int x, y, z;
    coords(c.G, p, x, y, z);
    if (i == 0) {
        const int ff = vfield<D>(cf), gf = vfield<D>(cg);
        Verts V = cell_verts<D>(c.G, x, y, z, 0, 0);
        const uint32_t t = crit_v(gf) ? vid(c.G, x + T.nb[ff][0], y + T.nb[ff][1], z + T.nb[ff][2]) : p;
        add_case<D>(c, t, V);
        return;
    }
    if (i <= T.NE) {
        const int e = i - 1;
        const int ff = efield<D>(cf, e), gf = efield<D>(cg, e);
        Verts V = cell_verts<D>(c.G, x, y, z, 1, e);
        uint32_t t;
        if (crit_c(gf))
            t = ff == 1 ? V.id[lowest_of(V, c.f)]
                        : vid(c.G, x + T.ecof_v[e][ff - 2][0], y + T.ecof_v[e][ff - 2][1], z + T.ecof_v[e][ff - 2][2]);
        else
            t = gf >= 2 ? V.id[lowest_of(V, c.f)] : fn_down_target<D>(c, x, y, z, 1, e, V);
        add_case<D>(c, t, V);
        return;
    }
    if (i <= T.NE + T.NT) {
        const int tt = i - 1 - T.NE;
        const int ff = tfield<D>(cf, tt), gf = tfield<D>(cg, tt);
        Verts V = cell_verts<D>(c.G, x, y, z, 2, tt);
        uint32_t t;
        if (crit_c(gf))
            t = ff == 1 ? V.id[lowest_of(V, c.f)]
                        : vid(c.G, x + T.tcof_v[tt][ff - 2][0], y + T.tcof_v[tt][ff - 2][1], z + T.tcof_v[tt][ff - 2][2]);
        else
            t = gf >= 2 ? V.id[lowest_of(V, c.f)] : fn_down_target<D>(c, x, y, z, 2, tt, V);
        add_case<D>(c, t, V);
        return;
    }
    const int k = i - 1 - T.NE - T.NT;
    const int gf = kfield<D>(cg, k);
    Verts V = cell_verts<D>(c.G, x, y, z, 3, k);
    const uint32_t t = crit_c(gf) ? V.id[lowest_of(V, c.f)] : fn_down_target<D>(c, x, y, z, 3, k, V);
    add_case<D>(c, t, V);
}

// ------------------------------------------------------------------------------------
// edit (Eq. 2) and dirty-anchor marking
// ------------------------------------------------------------------------------------
MSC_HD inline float clamp_base(float f, float fh, float xi)
{
    const float lb = sub_ru(f, xi), ub = add_rd(f, xi);
    return fh < lb ? lb : (fh > ub ? ub : fh);
}

// anchors whose code reads the value at v are v - o for the window offsets o; part/nparts
// split them among cooperating threads; each newly dirty anchor is handed to app (which
// appends it to the dirty list)
template <int D, class App> MSC_HD inline void mark_dirty(const Ctx &c, uint32_t v, int part, int nparts, App &&app)
{
    const Tab<D> &T = rt_tab<D>();
    int x, y, z;
    coords(c.G, v, x, y, z);
    for (int j = part; j < T.nwin; j += nparts) {
        const int px = x - T.win[j][0], py = y - T.win[j][1], pz = z - T.win[j][2];
        if (!inside(c.G, px, py, pz)) continue;
        const uint32_t p = vid(c.G, px, py, pz);
        if (!test_and_set(c.Dbits, p)) app(p);
    }
}

// Edit item i: i < nX restores Xlist[i] to f; otherwise Tlist[i - nX] takes a quantised
// step unless it is also restored or can no longer move.  Saves the vertex's value before
// the round in gprev (every item except a target that a restore item owns, so that gprev
// holds the pre-round value of every vertex in T u X) and returns whether the item changes
// its vertex, and the vertex.
MSC_HD inline bool edit_prepare(const Ctx &c, uint32_t i, uint32_t nX, uint32_t &v)
{
    if (i < nX) {
        v = c.Xlist[i];
        c.gprev[v] = c.g[v];
        return c.state[v] != ST_EXACT;
    }
    v = c.Tlist[i - nX];
    if ((c.Xbits[v >> 5] >> (v & 31)) & 1u) return false;
    c.gprev[v] = c.g[v];
    return c.state[v] <= c.qcap;
}

// Whether the round changed the SoS order of the edited vertex v against any vertex u
// within two edges of it (ring offsets `ring`, split among `nparts` cooperating threads).
// Every pair of vertices that a pairing rule compares lies within two edges (two
// neighbours of a vertex, two cofacet candidates of an edge or triangle, two vertices of a
// cell), so when no such order changes, no gradient code changes.  Values before the
// round: gprev for vertices in T u X (all saved by edit_prepare), g for the others.
template <int D>
MSC_HD inline bool order_changed(const Ctx &c, uint32_t v, int part, int nparts, const int (*ring)[3])
{
    const Tab<D> &T = rt_tab<D>();
    int x, y, z;
    coords(c.G, v, x, y, z);
    const float ov = c.gprev[v], nv = c.g[v];
    bool flip = false;
    for (int j = part; j < T.nring; j += nparts) {
        const int ux = x + ring[j][0], uy = y + ring[j][1], uz = z + ring[j][2];
        if (!inside(c.G, ux, uy, uz)) continue;
        const uint32_t u = vid(c.G, ux, uy, uz);
        const float nu = c.g[u];
        const bool moved = ((c.Tbits[u >> 5] | c.Xbits[u >> 5]) >> (u & 31)) & 1u;
        const float ou = moved ? c.gprev[u] : nu;
        flip |= sos_lt(ov, v, ou, u) != sos_lt(nv, v, nu, u);
    }
    return flip;
}

// Eq. 2 applied to a changing item: one step of xi / 2^q_max while q < q_max (q < qcap in
// floating-edit mode) and the value stays >= f - xi, otherwise the floor f - xi; a restore
// sets g = f exactly
// Eq. 2's step of target v from state st: the new value, and the new state in nst
MSC_HD inline float edit_value(const Ctx &c, uint32_t v, uint8_t st, uint8_t &nst)
{
    const float fv = ld(c.f + v);
    const float lb = sub_ru(fv, c.xi);
    if (st < c.qcap) {
        const float fc = clamp_base(fv, ld(c.fhat + v), c.xi);
        const float cand = sub_rn(fc, mul_rn((float)(st + 1), c.step));
        if (cand >= lb) { nst = (uint8_t)(st + 1); return cand; }
    }
    nst = ST_FLOOR;
    return lb;
}

// the edit of a new target by the C-pass thread that listed it (fuse_g set): the new value
// into fuse_g and the vertex onto the list of changed vertices; its state is left for the
// mark phase (state_after), so that every case of the round reads the pre-round state.  A
// target that a restore of the round also owns is restored after the C-pass, which wins.
MSC_HD inline void fuse_target(const Ctx &c, uint32_t t)
{
    const uint8_t st = c.state[t];
    if (st > c.qcap) return;            // at the floor or restored: nothing to change
    uint8_t nst;
    c.fuse_g[t] = edit_value(c, t, st, nst);
    c.Elist[list_slot(&c.cnt->nE)] = t;
}

// the state of a target that fuse_target edited in this round (not one a restore owns)
MSC_HD inline void state_after(const Ctx &c, uint32_t v)
{
    if ((c.Xbits[v >> 5] >> (v & 31)) & 1u) return;
    uint8_t nst;
    edit_value(c, v, c.state[v], nst);
    c.state[v] = nst;
}

MSC_HD inline void edit_apply(const Ctx &c, uint32_t i, uint32_t nX, uint32_t v)
{
    if (i < nX) {
        c.g[v] = ld(c.f + v);
        c.state[v] = ST_EXACT;
        return;
    }
    uint8_t nst;
    c.g[v] = edit_value(c, v, c.state[v], nst);
    c.state[v] = nst;
}

// one bit per cell the anchor owns: set if the cell is critical (tier 1: extrema only)
template <int D> MSC_HD inline uint64_t crit_sig(uint64_t code, int tier)
{
    constexpr int NE = Tab<D>::NE, NT = Tab<D>::NT, NK = Tab<D>::NK;
    uint64_t sig = (code & 15u) == 15u;
    if (tier >= 2 || D == 2) {
        // a 3-bit edge field is critical iff all its bits are 0 (likewise 2-bit triangle fields)
        if (tier >= 2) {
            const uint64_t e = code >> 4;
            uint64_t nz = 0;
            for (int i = 0; i < NE; i++) nz |= (uint64_t)(((e >> (3 * i)) & 7u) != 0) << i;
            sig |= (~nz & ((1ull << NE) - 1)) << 1;
        }
        const uint64_t t = code >> Tab<D>::TRI_BIT0;
        uint64_t nzt = 0;
        for (int i = 0; i < NT; i++) nzt |= (uint64_t)(((t >> (2 * i)) & 3u) != 0) << i;
        sig |= (~nzt & ((1ull << NT) - 1)) << (1 + NE);
    }
    const uint64_t k = code >> Tab<D>::TET_BIT0;
    sig |= (~k & ((1ull << NK) - 1)) << (1 + NE + NT);
    return sig;
}

// re-evaluate a dirty anchor (one pass)
template <int D> MSC_HD inline void refresh_anchor(const Ctx &c, uint32_t p)
{
    c.code_g[p] = anchor_code<D>(c.g, c.G, p);
}


// ------------------------------------------------------------------------------------
// S-pass (Sec. 4.4): walks along the separatrices of f, checked against g's gradient
// ------------------------------------------------------------------------------------
// descending path end (a minimum) of the V-path through vertex u in a gradient code
template <int D> MSC_HD inline uint32_t desc_end(const uint64_t *code, const Grid &G, uint32_t u)
{
    const Tab<D> &T = rt_tab<D>();
    int x, y, z;
    coords(G, u, x, y, z);
    for (uint32_t s = 0; s <= G.n; s++) {
        const int f = vfield<D>(ld(code + u));
        if (f == 15) return u;
        x += T.nb[f][0]; y += T.nb[f][1]; z += T.nb[f][2];
        u = vid(G, x, y, z);
    }
    return 0xFFFFFFFFu;
}

template <int D> MSC_HD inline void desc_walk_impl(const Ctx &c, uint32_t u, uint32_t &s)
{
    const Tab<D> &T = rt_tab<D>();
    int x, y, z;
    coords(c.G, u, x, y, z);
    for (s = 0; s <= c.G.n; s++) {
        if (test_and_set(c.vis_v, u)) return;
        const int ff = vfield<D>(ld(c.code_f + u));
        if (ff == 15) return;
        const int wx = x + T.nb[ff][0], wy = y + T.nb[ff][1], wz = z + T.nb[ff][2];
        const uint32_t w = vid(c.G, wx, wy, wz);
        if (vfield<D>(c.code_g[u]) != ff) {
            if (c.tier == 3 && desc_end<D>(c.code_f, c.G, u) == desc_end<D>(c.code_g, c.G, u)) return;
            Verts V;
            V.n = 0;
            vpush(V, c.G, x, y, z);
            vpush(V, c.G, wx, wy, wz);
            add_case<D>(c, w, V);
            return;
        }
        x = wx; y = wy; z = wz; u = w;
    }
}

template <int D> MSC_HD inline void desc_walk(const Ctx &c, uint32_t u)
{
    uint32_t s = 0;
    desc_walk_impl<D>(c, u, s);
    count_add(&c.cnt->steps[0], (unsigned long long)s + 1);
}

// top cells: tets (3D) or triangles (2D); id = anchor * NTOP + type
template <int D> MSC_HD inline int top_field(uint64_t code, int t) { return D == 3 ? kfield<D>(code, t) : tfield<D>(code, t); }
template <int D> MSC_HD inline Verts top_verts(const Grid &G, int x, int y, int z, int t)
{
    return cell_verts<D>(G, x, y, z, D == 3 ? 3 : 2, t);
}
template <int D> MSC_HD inline bool top_exists(const Grid &G, int x, int y, int z, int t)
{
    const Tab<D> &T = rt_tab<D>();
    const int top = D == 3 ? 7 : T.tB[t];
    return inside(G, x, y, z) && inside(G, x + (top & 1), y + ((top >> 1) & 1), z + ((top >> 2) & 1));
}

// one step of an ascending V-path: top cell (x,y,z,t) paired down (in the gradient "code"
// of field "vals") with its highest facet alpha; returns false if the cell is critical.
// Out: alpha's anchor/type, the index of the top cell in alpha's cofacet list, and the
// corner index (0..D) of the top cell's lowest vertex.
template <int D>
MSC_HD inline bool asc_facet(const Grid &G, const float *vals, int x, int y, int z, int t, const uint64_t *code,
                             int &fx, int &fy, int &fz, int &ft, int &ib, int &jlow)
{
    const Tab<D> &T = rt_tab<D>();
    if (top_field<D>(ld(code + vid(G, x, y, z)), t) == 0) return false;
    Verts V = top_verts<D>(G, x, y, z, t);
    jlow = lowest_of(V, vals);
    int corner;
    if (D == 3) corner = jlow == 0 ? 0 : (jlow == 1 ? T.kA[t] : (jlow == 2 ? T.kB[t] : 7));
    else corner = jlow == 0 ? 0 : (jlow == 1 ? T.tA[t] : T.tB[t]);
    int j = 0, ox, oy, oz;
    if (D == 3) {
        for (int q = 0; q < 4; q++) if (T.kfac_opp[t][q] == corner) j = q;
        ox = T.kfac_anc[t][j][0]; oy = T.kfac_anc[t][j][1]; oz = T.kfac_anc[t][j][2]; ft = T.kfac_type[t][j];
    } else {
        for (int q = 0; q < 3; q++) if (T.tfac_opp[t][q] == corner) j = q;
        ox = T.tfac_anc[t][j][0]; oy = T.tfac_anc[t][j][1]; oz = T.tfac_anc[t][j][2]; ft = T.tfac_type[t][j];
    }
    fx = x + ox; fy = y + oy; fz = z + oz;
    ib = -1;
    const int ncof = D == 3 ? T.ntcof[ft] : T.necof[ft];
    for (int i = 0; i < ncof; i++) {
        const int *an = D == 3 ? T.tcof_anc[ft][i] : T.ecof_anc[ft][i];
        const int ty = D == 3 ? T.tcof_type[ft][i] : T.ecof_type[ft][i];
        if (an[0] == -ox && an[1] == -oy && an[2] == -oz && ty == t) ib = i;
    }
    return true;
}

// the other top cofacet of facet (fx,fy,fz,ft) than cofacet index ib; false at the boundary
template <int D>
MSC_HD inline bool asc_next(const Grid &G, int fx, int fy, int fz, int ft, int ib, int &x, int &y, int &z, int &t)
{
    const Tab<D> &T = rt_tab<D>();
    const int ncof = D == 3 ? T.ntcof[ft] : T.necof[ft];
    if (ncof != 2) return false;
    const int io = 1 - ib;
    const int *an = D == 3 ? T.tcof_anc[ft][io] : T.ecof_anc[ft][io];
    x = fx + an[0]; y = fy + an[1]; z = fz + an[2];
    t = D == 3 ? T.tcof_type[ft][io] : T.ecof_type[ft][io];
    return top_exists<D>(G, x, y, z, t);
}

// field of a (D-1)-cell in a code
template <int D> MSC_HD inline int facet_field(uint64_t code, int ft) { return D == 3 ? tfield<D>(code, ft) : efield<D>(code, ft); }

// end of the ascending path entering top cell (x,y,z,t): (dim << 40) | cell id, where the
// cell id is anchor * NTOP + type for a maximum and anchor * 16 + type for a boundary facet
template <int D>
MSC_HD inline unsigned long long asc_end(const Grid &G, const float *vals, const uint64_t *code, int x, int y, int z, int t)
{
    const Tab<D> &T = rt_tab<D>();
    for (uint32_t s = 0; s <= G.n * (uint32_t)T.NTOP; s++) {
        int fx, fy, fz, ft, ib, jl;
        if (!asc_facet<D>(G, vals, x, y, z, t, code, fx, fy, fz, ft, ib, jl))
            return ((unsigned long long)D << 40) | ((unsigned long long)vid(G, x, y, z) * T.NTOP + t);
        if (!asc_next<D>(G, fx, fy, fz, ft, ib, x, y, z, t))
            return ((unsigned long long)(D - 1) << 40) | ((unsigned long long)vid(G, fx, fy, fz) * 16 + ft);
    }
    return ~0ull;
}

template <int D> MSC_HD inline void asc_walk_impl(const Ctx &c, uint32_t beta, uint32_t &s)
{
    const Tab<D> &T = rt_tab<D>();
    int x, y, z, t = (int)(beta % T.NTOP);
    coords(c.G, beta / T.NTOP, x, y, z);
    for (s = 0; s <= c.G.n * (uint32_t)T.NTOP; s++) {
        if (test_and_set(c.vis_top, vid(c.G, x, y, z) * T.NTOP + t)) return;
        int fx, fy, fz, ft, ib, jl;
        if (!asc_facet<D>(c.G, c.f, x, y, z, t, c.code_f, fx, fy, fz, ft, ib, jl)) return;   // maximum
        const int gf = facet_field<D>(c.code_g[vid(c.G, fx, fy, fz)], ft);
        if (gf != 2 + ib) {
            if (c.tier == 3 && asc_end<D>(c.G, c.f, c.code_f, x, y, z, t) == asc_end<D>(c.G, c.g, c.code_g, x, y, z, t))
                return;
            Verts V = top_verts<D>(c.G, x, y, z, t);
            add_case<D>(c, V.id[jl], V);
            return;
        }
        if (!asc_next<D>(c.G, fx, fy, fz, ft, ib, x, y, z, t)) return;   // leaves the domain
    }
}

template <int D> MSC_HD inline void asc_walk(const Ctx &c, uint32_t beta)
{
    uint32_t s = 0;
    asc_walk_impl<D>(c, beta, s);
    count_add(&c.cnt->steps[1], (unsigned long long)s + 1);
}

// saddle-saddle connectors (3D, tier 4): depth-first over triangles reached from a
// 2-saddle through edges paired upward in f; pairs missing from g's gradient are the
// troublemakers; a local stack spills to a global queue when full
constexpr int SS_STACK = 24;
constexpr unsigned TRI_LOCAL_STEPS = 512;   // per-thread saddle-saddle steps before the rest is spilled
                                           // (512^3 update: 64 steps 18.9 ms, 512 17.1, no limit 17.3)

MSC_HD inline void ss_push_global(const Ctx &c, uint32_t tri, uint32_t entry)
{
    const unsigned long long i = list_slot(&c.cnt->novf);
    if (i < c.ovf_cap) { c.ovf_out[2 * i] = tri; c.ovf_out[2 * i + 1] = entry; }
    else a_add(&c.cnt->err, 1ull);
}

// verification: record that the walk found a troublemaker among the facets of triangle tri
MSC_HD inline void ss_note_bad(const Ctx &c, uint32_t tri)
{
    if (!c.ss_bad || test_and_set(c.ss_bad, tri)) return;
    const unsigned long long i = list_slot(c.ss_n);
    if (i < c.ss_cap) c.ss_list[i] = tri;
    else a_add(&c.cnt->err, 1ull);
}

// start: (triangle id = anchor * 12 + type, entry edge id = anchor * 7 + type or ~0u);
// fresh seeds are marked visited here, spilled items were marked when first pushed
MSC_HD inline void ss_walk(const Ctx &c, uint32_t tri0, uint32_t entry0, bool seed)
{
    const Tab<3> &T = rt_tab<3>();
    if (seed && test_and_set(c.vis_tri, tri0)) return;
    uint32_t st_tri[SS_STACK], st_ent[SS_STACK];
    int sp = 0;
    unsigned long long nvis = 0;
    st_tri[sp] = tri0; st_ent[sp] = entry0; sp++;
    while (sp > 0) {
        sp--;
        nvis++;
        const uint32_t tri = st_tri[sp], entry = st_ent[sp];
        const int tt = (int)(tri % 12);
        int x, y, z;
        coords(c.G, tri / 12, x, y, z);
        for (int j = 0; j < 3; j++) {
            const int ex = x + T.tfac_anc[tt][j][0], ey = y + T.tfac_anc[tt][j][1], ez = z + T.tfac_anc[tt][j][2];
            const int et = T.tfac_type[tt][j];
            const uint32_t ea = vid(c.G, ex, ey, ez), eid = ea * 7 + (uint32_t)et;
            if (eid == entry) continue;
            const int ef = efield<3>(ld(c.code_f + ea), et);
            if (ef == 0) continue;                                   // 1-saddle: end
            const int eg = efield<3>(c.code_g[ea], et);
            if (ef == 1) {                                           // dead end in f
                if (eg != 1) {
                    Verts V = cell_verts<3>(c.G, ex, ey, ez, 1, et);
                    add_case<3>(c, V.id[lowest_of(V, c.f)], V);
                    ss_note_bad(c, tri);
                }
                continue;
            }
            const int i = ef - 2;
            const int tx = ex + T.ecof_anc[et][i][0], ty = ey + T.ecof_anc[et][i][1], tz = ez + T.ecof_anc[et][i][2];
            const int t2 = T.ecof_type[et][i];
            if (eg != ef) {
                Verts V = cell_verts<3>(c.G, tx, ty, tz, 2, t2);
                const uint32_t tv = vid(c.G, ex + T.ecof_v[et][i][0], ey + T.ecof_v[et][i][1], ez + T.ecof_v[et][i][2]);
                add_case<3>(c, tv, V);
                ss_note_bad(c, tri);
                continue;
            }
            const uint32_t tri2 = vid(c.G, tx, ty, tz) * 12 + (uint32_t)t2;
            if (tri2 == tri) continue;
            if (test_and_set(c.vis_tri, tri2)) continue;
            if (sp < SS_STACK) { st_tri[sp] = tri2; st_ent[sp] = eid; sp++; }
            else ss_push_global(c, tri2, eid);
        }
    }
    count_add(&c.cnt->steps[2], nvis);
}

// verification: a triangle t' = V_f(e) reached by the walk leads to a troublemaker, so do
// the reached triangles that cross into it: every reached triangle with facet e other than
// t' (its crossing (e, t') is the same pair, present in g since t' was reached).  e is the
// facet of t' opposite its f-lowest vertex.  A 2-saddle has no entry and no predecessor.
// Newly marked predecessors are appended to out.
MSC_HD inline void ss_back_step(const Ctx &c, uint32_t tri, uint32_t *out, unsigned long long *nout, uint32_t cap)
{
    const Tab<3> &T = rt_tab<3>();
    const int tt = (int)(tri % 12);
    int x, y, z;
    coords(c.G, tri / 12, x, y, z);
    if (tfield<3>(ld(c.code_f + tri / 12), tt) != 1) return;      // a 2-saddle (critical) root
    Verts V = cell_verts<3>(c.G, x, y, z, 2, tt);
    const int k = T.tri_opp[tt][lowest_of(V, c.f)];
    const int ex = x + T.tfac_anc[tt][k][0], ey = y + T.tfac_anc[tt][k][1], ez = z + T.tfac_anc[tt][k][2];
    const int et = T.tfac_type[tt][k];
    for (int i = 0; i < T.necof[et]; i++) {
        const int tx = ex + T.ecof_anc[et][i][0], ty = ey + T.ecof_anc[et][i][1], tz = ez + T.ecof_anc[et][i][2];
        const int t2 = T.ecof_type[et][i];
        const int top = T.tB[t2];
        if (!inside(c.G, tx, ty, tz) || !inside(c.G, tx + (top & 1), ty + ((top >> 1) & 1), tz + ((top >> 2) & 1)))
            continue;
        const uint32_t p = vid(c.G, tx, ty, tz) * 12 + (uint32_t)t2;
        if (p == tri) continue;
        if (!((c.vis_tri[p >> 5] >> (p & 31)) & 1u)) continue;     // not reached by the walk
        if (test_and_set(c.ss_bad, p)) continue;
        const unsigned long long j = list_slot(nout);
        if (j < cap) out[j] = p;
        else a_add(&c.cnt->err, 1ull);
    }
}

// ------------------------------------------------------------------------------------
// separatrix state (tier 4): the S-pass walks kept incrementally across S-passes
// ------------------------------------------------------------------------------------
// The S-pass of Sec. 4.4 walks every separatrix of f from its saddle and stops at the first
// pair missing from g's gradient.  The set of cells such a walk reaches depends on g only
// through the pairs it checks, and between two S-passes g changes only around edited
// vertices.  So the walks are kept as a state: one 16-bit word per node
//   descending: a vertex u (its pair (u, u next_f(u)));     ascending: a top cell beta (its
//   pair with its f-facet); saddle-saddle: a triangle t' = V_f(e) (pair (e, t')) and every
//   edge paired down in f (a dead end of the triangle walk);
// holding bit 0 = the node's f-pair is missing from g ("mismatch"), bit 1 = the node is a
// seed, bits 2.. = the signed number of reached predecessors passing into it.  A path node
// is reached iff it is a seed or has such a predecessor, and passes on iff reached and not
// mismatched; a triangle node passes on iff it is a seed, or has a reached parent and no
// mismatch.  Troublemakers are the mismatched nodes with a reached predecessor - exactly
// the first disagreeing pairs the walks stop at.  Every change is one atomic on the node's
// word and its before/after values decide the +-1 passed on, so concurrent updates settle
// on the same state in any order).
// Storage: two nodes per 32-bit word (node i in half i & 1), atomics on the word.  A node's
// count is kept with a bias, so a count that dips below zero while a +1 is in flight still
// leaves its half non-negative and never borrows from (or carries into) the other node:
// the biased field stays inside its 14 bits for counts in [-NS_BIAS, 2^14 - 1 - NS_BIAS].
// A fresh array is every byte NS_FILL (half 0x4040: no flags, count 0).  The helpers
// return a node decoded as an int32: flags in bits 0-1, the unbiased count in bits 2+.
constexpr int32_t NS_MIS = 1, NS_SEED = 2, NS_ONE = 4;
constexpr int32_t NS_BIAS = 0x1010;
constexpr int NS_FILL = 0x40;

__host__ __device__ constexpr size_t node_words(size_t nodes) { return (nodes + 1) / 2; }
MSC_HD inline int32_t node_decode(uint32_t word, uint32_t i)
{
    const int32_t h = (int32_t)((word >> ((i & 1u) * 16)) & 0xffffu);
    return (h & 3) | (((h >> 2) - NS_BIAS) * NS_ONE);
}

MSC_HD inline int32_t node_add(uint32_t *ns, uint32_t i, int delta)
{
    const uint32_t v = (uint32_t)(delta * NS_ONE) << ((i & 1u) * 16);
#ifdef __CUDA_ARCH__
    return node_decode(atomicAdd(ns + (i >> 1), v), i);
#else
    const uint32_t o = ns[i >> 1];
    ns[i >> 1] = o + v;
    return node_decode(o, i);
#endif
}

MSC_HD inline int32_t node_xor(uint32_t *ns, uint32_t i, int32_t m)
{
    const uint32_t v = (uint32_t)m << ((i & 1u) * 16);
#ifdef __CUDA_ARCH__
    return node_decode(atomicXor(ns + (i >> 1), v), i);
#else
    const uint32_t o = ns[i >> 1];
    ns[i >> 1] = o ^ v;
    return node_decode(o, i);
#endif
}

MSC_HD inline int32_t node_or(uint32_t *ns, uint32_t i, int32_t m)
{
    const uint32_t v = (uint32_t)m << ((i & 1u) * 16);
#ifdef __CUDA_ARCH__
    return node_decode(atomicOr(ns + (i >> 1), v), i);
#else
    const uint32_t o = ns[i >> 1];
    ns[i >> 1] = o | v;
    return node_decode(o, i);
#endif
}

MSC_HD inline int32_t node_load(const uint32_t *ns, uint32_t i)
{
    return node_decode(((const volatile uint32_t *)ns)[i >> 1], i);
}

MSC_HD inline int32_t node_count(int32_t b) { return b >> 2; }
MSC_HD inline bool path_reached(int32_t b) { return (b & NS_SEED) || node_count(b) > 0; }
MSC_HD inline int path_passes(int32_t b) { return path_reached(b) && !(b & NS_MIS); }
MSC_HD inline int tri_passes(int32_t b) { return (b & NS_SEED) || (node_count(b) > 0 && !(b & NS_MIS)); }

// successor of vertex u on its descending V-path in f
template <int D> MSC_HD inline bool desc_succ(const Ctx &c, uint32_t u, uint32_t &w)
{
    const Tab<D> &T = rt_tab<D>();
    const int ff = vfield<D>(ld(c.code_f + u));
    if (ff == 15) return false;
    if constexpr (D == 3) {
        // the lower neighbour a vertex is paired with is in the domain: no bounds to check
        const uint32_t b = ld(rt_tri_pack().nb + ff);
        w = u + (b & 3u) + ((b >> 2) & 3u) * (uint32_t)c.G.nx + ((b >> 4) & 3u) * (uint32_t)c.G.nx * (uint32_t)c.G.ny -
            (1u + (uint32_t)c.G.nx + (uint32_t)c.G.nx * (uint32_t)c.G.ny);
        return true;
    }
    int x, y, z;
    coords(c.G, u, x, y, z);
    w = vid(c.G, x + T.nb[ff][0], y + T.nb[ff][1], z + T.nb[ff][2]);
    return true;
}

// successor of top cell beta on its ascending V-path in f
template <int D> MSC_HD inline bool asc_succ(const Ctx &c, uint32_t beta, uint32_t &nb)
{
    if constexpr (D == 3) {
        // the tetrahedron's lowest vertex from the prepared slots: no vertex values to load
        const uint32_t a = beta / 6;
        const int t = (int)(beta % 6);
        const uint64_t cf = ld(c.code_f + a), lw = ld(c.low_f + a);
        if (kfield<3>(cf, t) == 0) return false;                 // a maximum
        const int jl = (int)((lw >> (24 + 2 * t)) & 3u);
        const uint32_t b = ld(&rt_tri_pack().asc[t][jl]);
        int x, y, z;
        coords(c.G, a, x, y, z);
        x += (int)(b & 3u) - 1; y += (int)((b >> 2) & 3u) - 1; z += (int)((b >> 4) & 3u) - 1;
        const int t2 = (int)((b >> 8) & 7u);
        if (!top_exists<3>(c.G, x, y, z, t2)) return false;      // the path leaves the domain
        nb = vid(c.G, x, y, z) * 6 + (uint32_t)t2;
        return true;
    }
    int x, y, z, t = (int)(beta % Tab<D>::NTOP);
    coords(c.G, beta / Tab<D>::NTOP, x, y, z);
    int fx, fy, fz, ft, ib, jl;
    if (!asc_facet<D>(c.G, c.f, x, y, z, t, c.code_f, fx, fy, fz, ft, ib, jl)) return false;
    if (!asc_next<D>(c.G, fx, fy, fz, ft, ib, x, y, z, t)) return false;
    nb = vid(c.G, x, y, z) * Tab<D>::NTOP + (uint32_t)t;
    return true;
}

// add delta to the reached-predecessor count of a path node and follow the change along
// the path (kind 0: descending vertices, 1: ascending top cells)
template <int D> MSC_HD inline void path_push(const Ctx &c, int kind, uint32_t w, int delta)
{
    uint32_t *ns = kind == 0 ? c.ns_v : c.ns_top;
    unsigned long long n = 0;
    for (uint32_t s = 0; s <= c.G.n * (uint32_t)Tab<D>::NTOP; s++) {
        n++;
        const int32_t o = node_add(ns, w, delta), nw = o + delta * NS_ONE;
        const int d = path_passes(nw) - path_passes(o);
        if (!d) break;
        uint32_t nx;
        if (!(kind == 0 ? desc_succ<D>(c, w, nx) : asc_succ<D>(c, w, nx))) break;
        w = nx;
        delta = d;
    }
    count_add(&c.cnt->steps[kind], n);
}

// a path node becomes a seed / changes its mismatch bit
template <int D> MSC_HD inline void path_change(const Ctx &c, int kind, uint32_t u, int32_t o, int32_t nw)
{
    const int d = path_passes(nw) - path_passes(o);
    uint32_t w;
    if (d && (kind == 0 ? desc_succ<D>(c, u, w) : asc_succ<D>(c, u, w))) path_push<D>(c, kind, w, d);
}

// children of a reached triangle node: its facet edges other than the one it is paired with
// in f; an edge paired up in f leads to its partner triangle, an edge paired down is a dead
// end, a critical edge (1-saddle) ends the walk.  One slot per facet edge j, so that every
// index is a constant and the slots stay in registers: kind[j] 0 (no child: the pair edge or
// a critical edge), 1 (a dead end: ch[j] is the edge id) or 2 (ch[j] is the partner triangle).
constexpr int TC_NONE = 0, TC_DEAD = 1, TC_LIVE = 2;
MSC_HD inline void tri_children(const Ctx &c, uint32_t tri, uint32_t (&ch)[3], int (&kind)[3])
{
    const TriPack &K = rt_tri_pack();
    const uint32_t a = tri / 12, tt = tri % 12;
    const uint32_t sy = (uint32_t)c.G.nx, sz = (uint32_t)c.G.nx * (uint32_t)c.G.ny;
    const uint32_t P = ld(K.tri + tt);
    int entry = -1;
    const uint64_t cf = ld(c.code_f + a), lw = ld(c.low_f + a);
    if (tfield<3>(cf, (int)tt) == 1) entry = (int)(P >> (24 + 2 * ((lw >> (2 * tt)) & 3u))) & 3;   // paired with the highest edge
#pragma unroll
    for (int j = 0; j < 3; j++) {
        kind[j] = TC_NONE;
        ch[j] = 0;
        if (j == entry) continue;
        // a facet or cofacet of a cell in the domain is in the domain: offsets need no bounds
        const uint32_t b = P >> (8 * j);
        const uint32_t ea = a + (b & 1u) + ((b >> 1) & 1u) * sy + ((b >> 2) & 1u) * sz;
        const int et = (int)((b >> 3) & 7u);
        const int ef = efield<3>(ld(c.code_f + ea), et);
        if (ef == 0) continue;
        if (ef == 1) { ch[j] = ea * 7 + (uint32_t)et; kind[j] = TC_DEAD; continue; }
        const uint32_t q = (uint32_t)(ld(K.ecof + et) >> (8 * (ef - 2)));
        ch[j] = (ea - (q & 1u) - ((q >> 1) & 1u) * sy - ((q >> 2) & 1u) * sz) * 12 + ((q >> 4) & 15u);
        kind[j] = TC_LIVE;
    }
}

MSC_HD inline void ss_spill(const Ctx &c, uint32_t tri, int delta)
{
    const unsigned long long i = list_slot(&c.cnt->novf);
    if (i < c.ovf_cap) { c.ovf_out[2 * i] = tri; c.ovf_out[2 * i + 1] = (uint32_t)delta; }
    else a_add(&c.cnt->err, 1ull);
}

// a triangle node's passing state changed by dv: pass dv to all its children, and keep
// following changes depth-first (local stack, spilled to a global queue when full)
MSC_HD inline void tri_propagate(const Ctx &c, uint32_t tri0, int dv0, bool apply_first, int delta0)
{
    uint32_t st[SS_STACK];
    int sd[SS_STACK];
    int sp = 0;
    unsigned long long n = 0;
    if (apply_first) { st[sp] = tri0; sd[sp] = delta0; sp++; }
    auto expand = [&](uint32_t t, int dv) {
        uint32_t ch[3];
        int kind[3];
        tri_children(c, t, ch, kind);
        for (int i = 0; i < 3; i++) {
            if (kind[i] == TC_DEAD) { node_add(c.ns_dead, ch[i], dv); continue; }
            if (kind[i] == TC_NONE) continue;
            if (sp < SS_STACK) { st[sp] = ch[i]; sd[sp] = dv; sp++; }
            else ss_spill(c, ch[i], dv);
        }
    };
    if (!apply_first) expand(tri0, dv0);
    while (sp > 0) {
#ifdef __CUDA_ARCH__
        // a long propagation goes on in the spill kernel, whose warps walk it converged: one
        // thread walking a large subtree alone would hold the whole launch
        if (n >= c.tri_local_steps) {
            for (int q = 0; q < sp; q++) ss_spill(c, st[q], sd[q]);
            break;
        }
#endif
        sp--;
        const uint32_t t = st[sp];
        const int d = sd[sp];
        n++;
        const int32_t o = node_add(c.ns_tri, t, d), nw = o + d * NS_ONE;
        const int dv = tri_passes(nw) - tri_passes(o);
        if (dv) expand(t, dv);
    }
    count_add(&c.cnt->steps[2], n);
}

// node states of the pairs anchored at p, from the codes of f and g.  init: only set the
// mismatch bits (all counts are zero); otherwise flip changed bits and propagate.
template <int D> MSC_HD inline void node_bits(const Ctx &c, uint32_t p, bool init)
{
    const Tab<D> &T = rt_tab<D>();
    const uint64_t cf = ld(c.code_f + p), cg = c.code_g[p];
    int x, y, z;
    coords(c.G, p, x, y, z);
    auto set_path = [&](int kind, uint32_t u, bool m) {
        uint32_t *ns = kind == 0 ? c.ns_v : c.ns_top;
        if (init) { if (m) node_or(ns, u, NS_MIS); return; }
        if (((node_load(ns, u) & NS_MIS) != 0) == m) return;
        const int32_t o = node_xor(ns, u, NS_MIS);
        path_change<D>(c, kind, u, o, o ^ NS_MIS);
    };
    const int vf = vfield<D>(cf);
    if (vf != 15) set_path(0, p, vfield<D>(cg) != vf);
    const int nfac = D == 3 ? T.NT : T.NE;
    for (int ft = 0; ft < nfac; ft++) {
        const int ff = facet_field<D>(cf, ft);
        if (ff < 2) continue;
        const int i = ff - 2;
        const int *an = D == 3 ? T.tcof_anc[ft][i] : T.ecof_anc[ft][i];
        const int bt = D == 3 ? T.tcof_type[ft][i] : T.ecof_type[ft][i];
        set_path(1, vid(c.G, x + an[0], y + an[1], z + an[2]) * T.NTOP + (uint32_t)bt, facet_field<D>(cg, ft) != ff);
    }
    if constexpr (D == 3) {
        for (int et = 0; et < T.NE; et++) {
            const int ef = efield<D>(cf, et);
            if (ef == 0) continue;
            const bool m = efield<D>(cg, et) != ef;
            if (ef == 1) {
                const uint32_t e = p * 7 + (uint32_t)et;
                if (init) { if (m) node_or(c.ns_dead, e, NS_MIS); continue; }
                if (((node_load(c.ns_dead, e) & NS_MIS) != 0) != m) node_xor(c.ns_dead, e, NS_MIS);
                continue;
            }
            const int i = ef - 2;
            const uint32_t t2 = vid(c.G, x + T.ecof_anc[et][i][0], y + T.ecof_anc[et][i][1], z + T.ecof_anc[et][i][2]) * 12 +
                                (uint32_t)T.ecof_type[et][i];
            if (init) { if (m) node_or(c.ns_tri, t2, NS_MIS); continue; }
            if (((node_load(c.ns_tri, t2) & NS_MIS) != 0) == m) continue;
            const int32_t o = node_xor(c.ns_tri, t2, NS_MIS);
            const int dv = tri_passes(o ^ NS_MIS) - tri_passes(o);
            if (dv) tri_propagate(c, t2, dv, false, 0);
        }
    }
}

// warp helpers that also compile for the host, where a "warp" is one lane (lane 0)
#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned warp_lane() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned warp_ballot(bool p) { return __ballot_sync(0xffffffffu, p); }
__device__ __forceinline__ bool warp_any(bool p) { return __any_sync(0xffffffffu, p); }
#else
inline unsigned warp_lane() { return 0; }
inline unsigned warp_ballot(bool p) { return p ? 1u : 0u; }
inline bool warp_any(bool p) { return p; }
#endif

// The first build's propagation along descending (kind 0) or ascending (kind 1) paths, with
// the lanes of a warp kept converged.  Every lane holds W slots; a slot is empty, a seed entry,
// or a walk at a node with the delta it passes on.  Empty slots are refilled together from the
// warp's current chunk of the seed list (a ballot and each lane's rank among the empty lanes,
// the same steps in every lane); then every slot does one operation in the same instruction
// stream: a seed entry sets its node's seed flag (atomic OR), a walk adds its delta (atomic
// add), and both fetch the node's f data for its successor beside the atomic.  A slot whose
// node starts to pass moves on to the successor; otherwise it empties.  A lane that walks
// alone while the others loop would leave most of the warp idle (an earlier form of this
// kernel ran at 3.3 active lanes per instruction).  The final node words are the same for any
// interleaving, as every change is an atomic whose before/after values decide what is passed
// on.  warp / nwarps: this warp's index and the number of warps; chunks of CH seeds are
// taken by warp, warp + nwarps, ...
template <int D, int W>
MSC_HD inline void path_seed_walks(const Ctx &c, int kind, const uint32_t *seeds, uint32_t n, unsigned long long warp,
                                   unsigned long long nwarps)
{
    const Tab<D> &T = rt_tab<D>();
    constexpr uint32_t NTOP = (uint32_t)Tab<D>::NTOP;
    constexpr unsigned long long CH = 256;            // seeds per warp chunk
    uint32_t *ns = kind == 0 ? c.ns_v : c.ns_top;
    const int64_t sy = c.G.nx, sz = (int64_t)c.G.nx * c.G.ny;
    const unsigned lt = (1u << warp_lane()) - 1u;
    unsigned long long cur = warp * CH, end = cur + CH < n ? cur + CH : n;
    bool more = cur < n;
    uint32_t node[W];
    int delta[W];
    int mode[W];                                      // 0 empty, 1 seed entry, 2 walk
    for (int k = 0; k < W; k++) { mode[k] = 0; node[k] = 0; delta[k] = 0; }
    unsigned long long steps = 0;
    for (;;) {
#pragma unroll
        for (int k = 0; k < W; k++) {
            unsigned em = warp_ballot(mode[k] == 0);
            while (em && more) {                      // warp-uniform
                const unsigned avail = (unsigned)(end - cur < 32 ? end - cur : 32);
                const unsigned cnt = (unsigned)__builtin_popcount(em);
                const unsigned take = cnt < avail ? cnt : avail;
                const unsigned rank = (unsigned)__builtin_popcount(em & lt);
                if (mode[k] == 0 && rank < take) {
                    node[k] = seeds[cur + rank];
                    mode[k] = 1;
                }
                cur += take;
                if (cur >= end) {
                    cur += (nwarps - 1) * CH;
                    end = cur + CH < n ? cur + CH : n;
                    more = cur < n;
                }
                em = warp_ballot(mode[k] == 0);
            }
        }
        bool busy = false;
        for (int k = 0; k < W; k++) busy = busy || mode[k] != 0;
        if (!warp_any(busy)) break;
        int32_t o[W];
        uint64_t cf[W], lw[W];
#pragma unroll
        for (int k = 0; k < W; k++) {
            o[k] = 0; cf[k] = 0; lw[k] = 0;
            if (mode[k] == 0) continue;
            const uint32_t a = kind == 0 ? node[k] : node[k] / NTOP;
            cf[k] = ld(c.code_f + a);
            if (D == 3 && kind == 1) lw[k] = ld(c.low_f + a);
            o[k] = mode[k] == 1 ? node_or(ns, node[k], NS_SEED) : node_add(ns, node[k], delta[k]);
        }
#pragma unroll
        for (int k = 0; k < W; k++) {
            if (mode[k] == 0) continue;
            int d;
            if (mode[k] == 1) {
                d = (o[k] & NS_SEED) ? 0 : path_passes(o[k] | NS_SEED) - path_passes(o[k]);
            } else {
                steps++;
                d = path_passes(o[k] + delta[k] * NS_ONE) - path_passes(o[k]);
            }
            bool cont = false;
            uint32_t w = 0;
            if (d) {
                if (kind == 0) {
                    const int ff = vfield<D>(cf[k]);
                    if (ff != 15) {
                        if constexpr (D == 3) {
                            const uint32_t b = ld(rt_tri_pack().nb + ff);
                            w = (uint32_t)((int64_t)node[k] + ((int)(b & 3u) - 1) + sy * ((int)((b >> 2) & 3u) - 1) +
                                           sz * ((int)((b >> 4) & 3u) - 1));
                        } else {
                            w = (uint32_t)((int64_t)node[k] + T.nb[ff][0] + sy * T.nb[ff][1] + sz * T.nb[ff][2]);
                        }
                        cont = true;
                    }
                } else if (D == 3) {
                    const uint32_t a = node[k] / NTOP;
                    const int t = (int)(node[k] % NTOP);
                    if (kfield<D>(cf[k], t) != 0) {
                        const int jl = (int)((lw[k] >> (24 + 2 * t)) & 3u);
                        const uint32_t b = ld(&rt_tri_pack().asc[t][jl]);
                        int x, y, z;
                        coords(c.G, a, x, y, z);
                        x += (int)(b & 3u) - 1; y += (int)((b >> 2) & 3u) - 1; z += (int)((b >> 4) & 3u) - 1;
                        const int t2 = (int)((b >> 8) & 7u);
                        if (top_exists<D>(c.G, x, y, z, t2)) {
                            w = vid(c.G, x, y, z) * NTOP + (uint32_t)t2;
                            cont = true;
                        }
                    }
                } else {
                    cont = asc_succ<D>(c, node[k], w);
                }
            }
            if (cont) { node[k] = w; delta[k] = d; mode[k] = 2; }
            else mode[k] = 0;
        }
    }
    count_add(&c.cnt->steps[kind], steps);
}

// The first build's saddle-saddle propagation with one stack per warp (in shared memory,
// `cap` entries): the lanes take up to 32 pending (triangle, delta) items at a time, apply
// them, and push the children that a change passes on back onto the warp's stack.  The
// lanes stay converged, where a depth-first walk per lane leaves most of them idle.  A full
// stack spills to the global queue that k_tri_spill drains.  Every change is an atomic on a
// node word, so the order of the items does not change the final state.  Must be called by
// whole warps; seeds are taken 32 at a time by each warp of the grid.  ITEMS: the list holds
// n (triangle, delta) pairs to apply (the spill queue) instead of seeds; they go onto the
// stack as they are.
template <bool ITEMS = false>
__device__ inline void tri_seed_walks(const Ctx &c, const uint32_t *seeds, uint32_t n, uint32_t *stk, int8_t *sdl, int cap)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long nwarps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    unsigned long long next = ((blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5) * 32;
    int sp = 0;                      // the same in every lane
    unsigned long long steps = 0;
    // push the live children of a triangle whose passing state changed by dv (lane-local
    // inputs; all lanes call it)
    auto push_children = [&](bool go, uint32_t t, int dv) {
        uint32_t ch[3] = {0, 0, 0};
        int kind[3] = {TC_NONE, TC_NONE, TC_NONE};
        if (go) tri_children(c, t, ch, kind);
#pragma unroll
        for (int r = 0; r < 3; r++) {
            const bool live = kind[r] == TC_LIVE;
            if (kind[r] == TC_DEAD) node_add(c.ns_dead, ch[r], dv);
            const unsigned m = __ballot_sync(0xffffffffu, live);
            const int cnt = __popc(m);
            if (!cnt) continue;
            const int pos = sp + __popc(m & ((1u << lane) - 1u));
            if (live) {
                if (pos < cap) { stk[pos] = ch[r]; sdl[pos] = (int8_t)dv; }
                else ss_spill(c, ch[r], dv);
            }
            sp = min(sp + cnt, cap);
        }
        __syncwarp();
    };
    for (;;) {
        if (sp < 32 && next < n) {
            // new seeds, one per lane: a 2-saddle triangle becomes a seed
            const unsigned long long i = next + lane;
            next += nwarps * 32;
            if constexpr (ITEMS) {
                const bool has = i < n;
                const uint32_t t = has ? seeds[2 * i] : 0u;
                const int d = has ? (int)seeds[2 * i + 1] : 0;
                const unsigned m = __ballot_sync(0xffffffffu, has);
                const int pos = sp + __popc(m & ((1u << lane) - 1u));
                if (has) {
                    if (pos < cap) { stk[pos] = t; sdl[pos] = (int8_t)d; }
                    else ss_spill(c, t, d);
                }
                sp = min(sp + __popc(m), cap);
                __syncwarp();
                continue;
            }
            bool go = false;
            int dv = 0;
            uint32_t u = 0;
            if (i < n) {
                u = seeds[i];
                const int32_t o = node_or(c.ns_tri, u, NS_SEED);
                if (!(o & NS_SEED)) {
                    dv = tri_passes(o | NS_SEED) - tri_passes(o);
                    go = dv != 0;
                }
            }
            push_children(go, u, dv);
            continue;
        }
        if (sp == 0) break;
        const int take = min(sp, 32);
        sp -= take;
        const bool act = (int)lane < take;
        uint32_t t = 0;
        int d = 0;
        if (act) { t = stk[sp + (int)lane]; d = sdl[sp + (int)lane]; }
        __syncwarp();
        bool go = false;
        int dv = 0;
        if (act) {
            steps++;
            const int32_t o = node_add(c.ns_tri, t, d), nw = o + d * NS_ONE;
            dv = tri_passes(nw) - tri_passes(o);
            go = dv != 0;
        }
        push_children(go, t, dv);
    }
    count_add(&c.cnt->steps[2], steps);
}

// Troublemakers (Sec. 4.4) at a mismatched anchor p, one pair field at a time.  Field i:
// 0 the vertex's pair, 1 + ft the pair of facet ft (tri in 3D, edge in 2D) with its top
// cofacet, 1 + NFAC + et (3D) the pair of edge et with its triangle (or a dead end).
// node_target_mask: bit i set iff field i is paired in f and differs in g (only those
// nodes carry the mismatch bit, so only they are read).
template <int D> MSC_HD inline uint32_t node_target_mask(uint64_t cf, uint64_t cg)
{
    const Tab<D> &T = rt_tab<D>();
    if (cf == cg) return 0;
    uint32_t m = 0;
    const int vf = vfield<D>(cf);
    if (vf != 15 && vfield<D>(cg) != vf) m |= 1u;
    const int nfac = D == 3 ? T.NT : T.NE;
    for (int ft = 0; ft < nfac; ft++) {
        const int ff = facet_field<D>(cf, ft);
        if (ff >= 2 && facet_field<D>(cg, ft) != ff) m |= 1u << (1 + ft);
    }
    if constexpr (D == 3)
        for (int et = 0; et < T.NE; et++) {
            const int ef = efield<D>(cf, et);
            if (ef != 0 && efield<D>(cg, et) != ef) m |= 1u << (1 + nfac + et);
        }
    return m;
}

template <int D> MSC_HD inline void node_target_item(const Ctx &c, uint32_t p, uint64_t cf, int i)
{
    const Tab<D> &T = rt_tab<D>();
    constexpr int NFAC = D == 3 ? Tab<D>::NT : Tab<D>::NE;
    int x, y, z;
    coords(c.G, p, x, y, z);
    if (i == 0) {
        const int vf = vfield<D>(cf);
        const int32_t b = node_load(c.ns_v, p);
        if ((b & NS_MIS) && path_reached(b)) {
            Verts V;
            V.n = 0;
            vpush(V, c.G, x, y, z);
            vpush(V, c.G, x + T.nb[vf][0], y + T.nb[vf][1], z + T.nb[vf][2]);
            add_case<D>(c, V.id[1], V);
        }
        return;
    }
    if (i <= NFAC) {
        const int ft = i - 1;
        const int ff = facet_field<D>(cf, ft);
        const int k = ff - 2;
        const int *an = D == 3 ? T.tcof_anc[ft][k] : T.ecof_anc[ft][k];
        const int bt = D == 3 ? T.tcof_type[ft][k] : T.ecof_type[ft][k];
        const int bx = x + an[0], by = y + an[1], bz = z + an[2];
        const int32_t b = node_load(c.ns_top, vid(c.G, bx, by, bz) * T.NTOP + (uint32_t)bt);
        if ((b & NS_MIS) && path_reached(b)) {
            Verts V = top_verts<D>(c.G, bx, by, bz, bt);
            add_case<D>(c, V.id[lowest_of(V, c.f)], V);
        }
        return;
    }
    if constexpr (D == 3) {
        const int et = i - 1 - NFAC;
        const int ef = efield<D>(cf, et);
        if (ef == 1) {
            const int32_t b = node_load(c.ns_dead, p * 7 + (uint32_t)et);
            if ((b & NS_MIS) && node_count(b) > 0) {
                Verts V = cell_verts<3>(c.G, x, y, z, 1, et);
                add_case<3>(c, V.id[lowest_of(V, c.f)], V);
            }
            return;
        }
        const int k = ef - 2;
        const int tx = x + T.ecof_anc[et][k][0], ty = y + T.ecof_anc[et][k][1], tz = z + T.ecof_anc[et][k][2];
        const int t2 = T.ecof_type[et][k];
        const int32_t b = node_load(c.ns_tri, vid(c.G, tx, ty, tz) * 12 + (uint32_t)t2);
        if ((b & NS_MIS) && node_count(b) > 0 && !(b & NS_SEED)) {
            Verts V = cell_verts<3>(c.G, tx, ty, tz, 2, t2);
            add_case<3>(c, vid(c.G, x + T.ecof_v[et][k][0], y + T.ecof_v[et][k][1], z + T.ecof_v[et][k][2]), V);
        }
    }
}

// all troublemakers at anchor p
template <int D> MSC_HD inline void node_targets(const Ctx &c, uint32_t p)
{
    const uint64_t cf = ld(c.code_f + p), cg = c.code_g[p];
    for (int i = 0; i < 32; i++)
        if ((node_target_mask<D>(cf, cg) >> i) & 1u) node_target_item<D>(c, p, cf, i);
}

// ------------------------------------------------------------------------------------
// seeds of the separatrices of f (once per original field)
// ------------------------------------------------------------------------------------
// kind 0: descending seeds (both vertices of every critical edge); kind 1: ascending seeds
// (top cofacets of every critical (D-1)-cell); kind 2: 2-saddle triangles (3D)
template <int D, class Emit> MSC_HD inline void seeds_of_code(uint64_t cf, const Grid &G, uint32_t p, int x, int y, int z,
                                                              int kind, Emit &&emit)
{
    using Tb = Tab<D>;
    const unsigned cin = corner_mask<D>(G, x, y, z);
    if (kind == 0 || (D == 2 && kind == 1)) {
        static_for<Tb::NE>([&](auto ec) {
            constexpr int e = decltype(ec)::value;
            if (!((cin >> (e + 1)) & 1u) || efield<D>(cf, e) != 0) return;
            if (kind == 0) {
                constexpr int A = e + 1;
                emit(p);
                emit(vid(G, x + (A & 1), y + ((A >> 1) & 1), z + ((A >> 2) & 1)));
                return;
            }
            static_for<TabC<D>::T.necof[e]>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int ax = TabC<D>::T.ecof_anc[e][i][0], ay = TabC<D>::T.ecof_anc[e][i][1];
                constexpr int az = TabC<D>::T.ecof_anc[e][i][2], bt = TabC<D>::T.ecof_type[e][i];
                if (top_exists<D>(G, x + ax, y + ay, z + az, bt)) emit(vid(G, x + ax, y + ay, z + az) * Tb::NTOP + bt);
            });
        });
        return;
    }
    if constexpr (D == 3) {
        static_for<Tb::NT>([&](auto tc) {
            constexpr int tt = decltype(tc)::value;
            constexpr int top = TabC<D>::T.tB[tt];
            if (!((cin >> top) & 1u) || tfield<D>(cf, tt) != 0) return;
            if (kind == 2) {
                emit(p * 12 + tt);
                return;
            }
            static_for<TabC<D>::T.ntcof[tt]>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int ax = TabC<D>::T.tcof_anc[tt][i][0], ay = TabC<D>::T.tcof_anc[tt][i][1];
                constexpr int az = TabC<D>::T.tcof_anc[tt][i][2], bt = TabC<D>::T.tcof_type[tt][i];
                if (top_exists<D>(G, x + ax, y + ay, z + az, bt)) emit(vid(G, x + ax, y + ay, z + az) * Tb::NTOP + bt);
            });
        });
    }
}

// the separatrix seeds of f that anchor p owns, by kind (see seeds_of_code)
template <int D, class Emit> MSC_HD inline void seeds_anchor(const uint64_t *code, const Grid &G, uint32_t p, int kind,
                                                             Emit &&emit)
{
    int x, y, z;
    coords(G, p, x, y, z);
    seeds_of_code<D>(ld(code + p), G, p, x, y, z, kind, emit);
}

// ------------------------------------------------------------------------------------
// decoding a code into canonical vertex tuples (introspection and verification)
// ------------------------------------------------------------------------------------
MSC_HD inline void sort4(int64_t *r, int n)
{
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && r[j - 1] > r[j]; j--) { int64_t t = r[j]; r[j] = r[j - 1]; r[j - 1] = t; }
    for (int i = n; i < 4; i++) r[i] = -1;
}

// pairs (L, U) with L owned by anchor p and paired upward: rows of 8 ids
template <int D> MSC_HD inline void decode_pairs(const uint64_t *code, const Grid &G, uint32_t p, int64_t *rows,
                                                 unsigned long long *count, unsigned long long cap)
{
    const Tab<D> &T = rt_tab<D>();
    int x, y, z;
    coords(G, p, x, y, z);
    const unsigned cin = corner_mask<D>(G, x, y, z);
    const uint64_t cf = ld(code + p);
    auto emit = [&](const Verts &L, int ex, int ey, int ez) {
        const unsigned long long i = list_slot(count);
        if (!rows || i >= cap) return;
        int64_t *r = rows + 8 * i;
        for (int k = 0; k < L.n; k++) { r[k] = L.id[k]; r[4 + k] = L.id[k]; }
        sort4(r, L.n);
        r[4 + L.n] = vid(G, ex, ey, ez);
        sort4(r + 4, L.n + 1);
    };
    const int vf = vfield<D>(cf);
    if (vf != 15) emit(cell_verts<D>(G, x, y, z, 0, 0), x + T.nb[vf][0], y + T.nb[vf][1], z + T.nb[vf][2]);
    for (int e = 0; e < T.NE; e++) {
        const int f = efield<D>(cf, e);
        if (!((cin >> (e + 1)) & 1u) || f < 2) continue;
        emit(cell_verts<D>(G, x, y, z, 1, e), x + T.ecof_v[e][f - 2][0], y + T.ecof_v[e][f - 2][1], z + T.ecof_v[e][f - 2][2]);
    }
    for (int tt = 0; tt < T.NT; tt++) {
        const int f = tfield<D>(cf, tt);
        if (!((cin >> T.tB[tt]) & 1u) || f < 2) continue;
        emit(cell_verts<D>(G, x, y, z, 2, tt), x + T.tcof_v[tt][f - 2][0], y + T.tcof_v[tt][f - 2][1], z + T.tcof_v[tt][f - 2][2]);
    }
}

// critical cells owned by anchor p: rows of 4 ids + dimension.  If ref != nullptr, count
// instead the cells whose criticality differs from ref's (fp: critical only in code,
// fn: critical only in ref) into cnt->rep[dim] / rep[4 + dim]
template <int D> MSC_HD inline void decode_critical(const uint64_t *code, const uint64_t *ref, const Grid &G, uint32_t p,
                                                    int64_t *rows, int32_t *dims, unsigned long long *count,
                                                    unsigned long long cap, Counters *cnt)
{
    const Tab<D> &T = rt_tab<D>();
    int x, y, z;
    coords(G, p, x, y, z);
    const unsigned cin = corner_mask<D>(G, x, y, z);
    const uint64_t cf = ld(code + p);
    const uint64_t rf = ref ? ld(ref + p) : 0;
    auto handle = [&](bool crit, bool rcrit, int kind, int t) {
        if (ref) {
            if (crit && !rcrit) a_add(&cnt->rep[kind], 1ull);
            if (!crit && rcrit) a_add(&cnt->rep[4 + kind], 1ull);
            return;
        }
        if (!crit) return;
        const unsigned long long i = list_slot(count);
        if (!rows || i >= cap) return;
        Verts V = cell_verts<D>(G, x, y, z, kind, t);
        for (int k = 0; k < V.n; k++) rows[4 * i + k] = V.id[k];
        sort4(rows + 4 * i, V.n);
        dims[i] = kind;
    };
    handle(vfield<D>(cf) == 15, vfield<D>(rf) == 15, 0, 0);
    for (int e = 0; e < T.NE; e++)
        if ((cin >> (e + 1)) & 1u) handle(efield<D>(cf, e) == 0, efield<D>(rf, e) == 0, 1, e);
    for (int tt = 0; tt < T.NT; tt++)
        if ((cin >> T.tB[tt]) & 1u) handle(tfield<D>(cf, tt) == 0, tfield<D>(rf, tt) == 0, 2, tt);
    for (int k = 0; k < T.NK; k++)
        if ((cin >> 7) & 1u) handle(kfield<D>(cf, k) == 0, kfield<D>(rf, k) == 0, 3, k);
}

}  // namespace msc
