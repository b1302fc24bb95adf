// Cell tables of the Freudenthal triangulation and the per-anchor discrete-gradient
// evaluator used by every kernel of libmsc.
//
// Every cell of the triangulated grid is owned by its anchor: its smallest-index vertex p.
// Relative to p its vertices are p + e_S for a chain of axis sets 0 = S0 < S1 < ... (S a
// bitmask over x=1, y=2, z=4); "corner k" of the cube at p is p + e_k.  A 3D anchor owns
// 1 vertex, 7 edges, 12 triangles and 6 tetrahedra (Sec. 4.8.1: N1 ~ 7N0, N2 ~ 12N0,
// N3 ~ 6N0); a 2D anchor owns 1 vertex, 3 edges and 2 triangles.
//
// The gradient of all cells an anchor owns is packed into one 64-bit code per vertex
// (this build's form of the per-cell lookup codes of Sec. 4.8.1):
//   bits [0,4)                vertex: neighbour index 0..NNB-1 of its pair edge, 15 = critical
//   3 bits per edge           0 critical, 1 paired down (with its higher vertex),
//                             2+i paired up with cofacet triangle i of the edge type
//   2 bits per triangle       0 critical, 1 paired down, 2+i paired up with cofacet tet i
//   1 bit per tetrahedron     0 critical, 1 paired down
// (3D: 4 + 21 + 24 + 6 = 55 bits; 2D: 4 + 9 + 4 = 17 bits.)  Cells that do not exist
// (anchor on the upper boundary) have all-zero fields in every code.
//
// All tables are computed at compile time from the chain definition, so that loops over
// cell types unroll into straight-line code with immediate window offsets.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>

#ifdef MSC_HOST_EMULATION
#define MSC_HD __host__ __device__
#else
#define MSC_HD __device__
#endif

namespace msc {

#ifdef __CUDA_ARCH__
__device__ __forceinline__ float pos_inf() { return __int_as_float(0x7f800000); }
#else
inline float pos_inf() { return __builtin_huge_valf(); }
#endif

// window of g around an anchor: offsets in [-1, 2]^D, index (x+1) + 4(y+1) + 16(z+1);
// the index order equals the vertex-id order of any two in-domain positions.
template <int D> struct Tab {
    static constexpr int AX = D == 3 ? 7 : 3;     // full axis mask
    static constexpr int NC = D == 3 ? 8 : 4;     // cube corners
    static constexpr int NNB = D == 3 ? 14 : 6;   // neighbours of a vertex
    static constexpr int NE = D == 3 ? 7 : 3;     // edges per anchor
    static constexpr int NT = D == 3 ? 12 : 2;    // triangles per anchor
    static constexpr int NK = D == 3 ? 6 : 0;     // tetrahedra per anchor
    static constexpr int NCE = D == 3 ? 19 : 5;   // edges of the cube at an anchor
    static constexpr int NCT = D == 3 ? 18 : 2;   // triangles of the cube at an anchor
    static constexpr int NTOP = D == 3 ? 6 : 2;   // top cells per anchor
    static constexpr int WS = D == 3 ? 64 : 16;   // window size
    static constexpr int TRI_BIT0 = 4 + 3 * NE;
    static constexpr int TET_BIT0 = TRI_BIT0 + 2 * NT;

    int nb[14][3];                 // neighbour offsets: n < NE: +e_{n+1}; else -e_{n-NE+1}
    int tA[12], tB[12];            // triangle type t: corners {0, tA, tB}
    int kA[6], kB[6];              // tet type t: corners {0, kA, kB, AX}
    int necof[7];                  // cofacets of edge type t
    int ecof_v[7][6][3];           //   extra vertex offset (relative to the edge's anchor)
    int ecof_anc[7][6][3];         //   anchor offset of the cofacet triangle
    int ecof_type[7][6];           //   its triangle type
    int ntcof[12];                 // cofacets of triangle type t
    int tcof_v[12][2][3], tcof_anc[12][2][3], tcof_type[12][2];
    int tfac_anc[12][3][3], tfac_type[12][3], tfac_opp[12][3];  // facet edge j, opposite corner
    int kfac_anc[6][4][3], kfac_type[6][4], kfac_opp[6][4];     // facet triangle j, opposite corner
    // dense evaluator: window positions
    int cpos[8];                   // corner k
    int cnb[8][14];                // corner k + nb[n]
    int cnb_ord[8][14];            // neighbour indices n of corner k by increasing window position
    int nwin;                      // window offsets an anchor's code reads: [-1,1]^D u [0,2]^D
    int win[64][3];
    int ce_a[19], ce_b[19];        // cube edges: corners a < b (a subset of b)
    int ce_cof[19][6];             // window positions of the cofacet extra vertices
    int ce_ncof[19];
    int ct_a[18], ct_b[18], ct_c[18];      // cube triangles: corners a < b < c
    int ct_e[18][3];               // cube-edge index of edges (a,b), (a,c), (b,c)
    int ct_opp_pos[18][3];         // position of the opposite corner in that edge's cofacet list
    int ct_cof[18][2], ct_ncof[18];
    int k_tri[6][4];               // tet t: cube-triangle index of the facet opposite corner
                                   //   0, kA, kB, AX (in that order)
    int k_opp_pos[6][4];           // position of that corner in the facet's cofacet list
    // vertices within two edges of a vertex (sums of at most two neighbour offsets, the
    // vertex itself excluded): every pair of vertices whose SoS order the pairing rules
    // compare lies in one such set (neighbours of a vertex, cofacet candidates of an edge
    // or triangle, vertices of a cell)
    int nring;
    int ring[64][3];
    // ascending V-path step in f (Sec. 4.4): a top cell of type t paired with its highest
    // facet (the one opposite its lowest vertex, slot j in cell order) continues into that
    // facet's other cofacet, of type asc_type[t][j] at anchor offset asc_off[t][j]
    int asc_off[6][4][3];
    int asc_type[6][4];
    // triangle type t whose lowest vertex is slot j: the index of the facet edge opposite it
    int tri_opp[12][3];
};

constexpr int popc3(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1); }
template <int D> constexpr int wpos(int x, int y, int z) { return (x + 1) + 4 * (y + 1) + (D == 3 ? 16 * (z + 1) : 0); }

template <int D> constexpr int tri_type_of(int A, int B)
{
    int t = 0;
    for (int b = 1; b <= Tab<D>::AX; b++)
        for (int a = 1; a <= Tab<D>::AX; a++)
            if ((a & b) == a && a != b && (b & ~Tab<D>::AX) == 0) {
                if (a == A && b == B) return t;
                t++;
            }
    return -1;
}

template <int D> constexpr int tet_type_of(int A, int B)
{
    int t = 0;
    for (int b = 1; b <= 7; b++) {
        if (popc3(b) != 2) continue;
        for (int a = 1; a <= 7; a++) {
            if (popc3(a) != 1 || (a & b) != a) continue;
            if (a == A && b == B) return t;
            t++;
        }
    }
    return -1;
}

constexpr bool adjacent_off(int ux, int uy, int uz, int vx, int vy, int vz)
{
    int dx = vx - ux, dy = vy - uy, dz = vz - uz;
    if (dx == 0 && dy == 0 && dz == 0) return false;
    bool pos = dx >= 0 && dy >= 0 && dz >= 0 && dx <= 1 && dy <= 1 && dz <= 1;
    bool neg = dx <= 0 && dy <= 0 && dz <= 0 && dx >= -1 && dy >= -1 && dz >= -1;
    return pos || neg;
}

// a cell given by n vertex offsets -> (anchor offset, type); returns false if not a cell
template <int D> constexpr bool normalize(const int (*v)[3], int n, int anc[3], int &type)
{
    int lo = 0;
    for (int i = 1; i < n; i++) {
        const int *a = v[i], *b = v[lo];
        if (a[2] < b[2] || (a[2] == b[2] && (a[1] < b[1] || (a[1] == b[1] && a[0] < b[0])))) lo = i;
    }
    anc[0] = v[lo][0]; anc[1] = v[lo][1]; anc[2] = v[lo][2];
    int m[4] = {0, 0, 0, 0}, k = 0;
    for (int i = 0; i < n; i++) {
        if (i == lo) continue;
        int dx = v[i][0] - anc[0], dy = v[i][1] - anc[1], dz = v[i][2] - anc[2];
        if (dx < 0 || dy < 0 || dz < 0 || dx > 1 || dy > 1 || dz > 1) return false;
        m[k++] = dx | (dy << 1) | (dz << 2);
    }
    for (int i = 1; i < k; i++)           // sort by size: a chain is totally ordered
        for (int j = i; j > 0 && popc3(m[j - 1]) > popc3(m[j]); j--) { int t = m[j]; m[j] = m[j - 1]; m[j - 1] = t; }
    for (int i = 1; i < k; i++)
        if ((m[i - 1] & m[i]) != m[i - 1] || m[i - 1] == m[i]) return false;
    if (n == 2) type = m[0] - 1;
    else if (n == 3) type = tri_type_of<D>(m[0], m[1]);
    else if (n == 4) type = tet_type_of<D>(m[0], m[1]);
    else type = 0;
    return type >= 0;
}

template <int D> constexpr Tab<D> make_tab()
{
    using T = Tab<D>;
    Tab<D> t{};
    for (int n = 0; n < T::NE; n++) {
        int A = n + 1;
        t.nb[n][0] = A & 1; t.nb[n][1] = (A >> 1) & 1; t.nb[n][2] = (A >> 2) & 1;
        t.nb[n + T::NE][0] = -(A & 1); t.nb[n + T::NE][1] = -((A >> 1) & 1); t.nb[n + T::NE][2] = -((A >> 2) & 1);
    }
    {
        int k = 0;
        for (int b = 1; b <= T::AX; b++)
            for (int a = 1; a <= T::AX; a++)
                if ((a & b) == a && a != b) { t.tA[k] = a; t.tB[k] = b; k++; }
        k = 0;
        if (D == 3)
            for (int b = 1; b <= 7; b++) {
                if (popc3(b) != 2) continue;
                for (int a = 1; a <= 7; a++)
                    if (popc3(a) == 1 && (a & b) == a) { t.kA[k] = a; t.kB[k] = b; k++; }
            }
    }
    const int zlo = D == 3 ? -1 : 0, zhi = D == 3 ? 2 : 0;
    // edge-type cofacets: third vertices adjacent to both ends, in window order
    for (int e = 0; e < T::NE; e++) {
        int A = e + 1, ax = A & 1, ay = (A >> 1) & 1, az = (A >> 2) & 1, n = 0;
        for (int z = zlo; z <= zhi; z++)
            for (int y = -1; y <= 2; y++)
                for (int x = -1; x <= 2; x++) {
                    if (!adjacent_off(0, 0, 0, x, y, z) || !adjacent_off(ax, ay, az, x, y, z)) continue;
                    int v[3][3] = {{0, 0, 0}, {ax, ay, az}, {x, y, z}}, anc[3] = {0, 0, 0}, ty = -1;
                    if (!normalize<D>(v, 3, anc, ty)) continue;
                    t.ecof_v[e][n][0] = x; t.ecof_v[e][n][1] = y; t.ecof_v[e][n][2] = z;
                    t.ecof_anc[e][n][0] = anc[0]; t.ecof_anc[e][n][1] = anc[1]; t.ecof_anc[e][n][2] = anc[2];
                    t.ecof_type[e][n] = ty;
                    n++;
                }
        t.necof[e] = n;
    }
    // triangle types: cofacets and facets
    for (int tt = 0; tt < T::NT; tt++) {
        int A = t.tA[tt], B = t.tB[tt];
        int v[3][3] = {{0, 0, 0}, {A & 1, (A >> 1) & 1, (A >> 2) & 1}, {B & 1, (B >> 1) & 1, (B >> 2) & 1}};
        int n = 0;
        for (int z = zlo; z <= zhi; z++)
            for (int y = -1; y <= 2; y++)
                for (int x = -1; x <= 2; x++) {
                    bool ok = true;
                    for (int i = 0; i < 3; i++) ok = ok && adjacent_off(v[i][0], v[i][1], v[i][2], x, y, z);
                    if (!ok) continue;
                    int w[4][3] = {{v[0][0], v[0][1], v[0][2]}, {v[1][0], v[1][1], v[1][2]},
                                   {v[2][0], v[2][1], v[2][2]}, {x, y, z}};
                    int anc[3] = {0, 0, 0}, ty = -1;
                    if (!normalize<D>(w, 4, anc, ty)) continue;
                    t.tcof_v[tt][n][0] = x; t.tcof_v[tt][n][1] = y; t.tcof_v[tt][n][2] = z;
                    t.tcof_anc[tt][n][0] = anc[0]; t.tcof_anc[tt][n][1] = anc[1]; t.tcof_anc[tt][n][2] = anc[2];
                    t.tcof_type[tt][n] = ty;
                    n++;
                }
        t.ntcof[tt] = n;
        const int corner[3] = {0, A, B};
        for (int j = 0; j < 3; j++) {         // facet j = triangle minus vertex j
            int w[2][3] = {}, m = 0;
            for (int i = 0; i < 3; i++)
                if (i != j) { w[m][0] = v[i][0]; w[m][1] = v[i][1]; w[m][2] = v[i][2]; m++; }
            int anc[3] = {0, 0, 0}, ty = -1;
            normalize<D>(w, 2, anc, ty);
            t.tfac_anc[tt][j][0] = anc[0]; t.tfac_anc[tt][j][1] = anc[1]; t.tfac_anc[tt][j][2] = anc[2];
            t.tfac_type[tt][j] = ty;
            t.tfac_opp[tt][j] = corner[j];
        }
    }
    for (int kk = 0; kk < T::NK; kk++) {
        int A = t.kA[kk], B = t.kB[kk];
        const int corner[4] = {0, A, B, 7};
        int v[4][3] = {};
        for (int i = 0; i < 4; i++) { v[i][0] = corner[i] & 1; v[i][1] = (corner[i] >> 1) & 1; v[i][2] = (corner[i] >> 2) & 1; }
        for (int j = 0; j < 4; j++) {
            int w[3][3] = {}, m = 0;
            for (int i = 0; i < 4; i++)
                if (i != j) { w[m][0] = v[i][0]; w[m][1] = v[i][1]; w[m][2] = v[i][2]; m++; }
            int anc[3] = {0, 0, 0}, ty = -1;
            normalize<D>(w, 3, anc, ty);
            t.kfac_anc[kk][j][0] = anc[0]; t.kfac_anc[kk][j][1] = anc[1]; t.kfac_anc[kk][j][2] = anc[2];
            t.kfac_type[kk][j] = ty;
            t.kfac_opp[kk][j] = corner[j];
        }
    }
    t.nring = 0;
    for (int a = -1; a < T::NNB; a++)
        for (int b = a; b < T::NNB; b++) {
            int o[3] = {0, 0, 0};
            for (int i = 0; i < 3; i++) o[i] = (a >= 0 ? t.nb[a][i] : 0) + (b >= 0 ? t.nb[b][i] : 0);
            if (o[0] == 0 && o[1] == 0 && o[2] == 0) continue;
            bool seen = false;
            for (int k = 0; k < t.nring; k++)
                if (t.ring[k][0] == o[0] && t.ring[k][1] == o[1] && t.ring[k][2] == o[2]) seen = true;
            if (seen) continue;
            t.ring[t.nring][0] = o[0]; t.ring[t.nring][1] = o[1]; t.ring[t.nring][2] = o[2];
            t.nring++;
        }
    for (int tt = 0; tt < T::NTOP; tt++) {
        const int nv = D + 1;
        const int cs[4] = {0, D == 3 ? t.kA[tt] : t.tA[tt], D == 3 ? t.kB[tt] : t.tB[tt], 7};
        for (int j = 0; j < nv; j++) {
            int fj = 0;
            for (int q = 0; q < nv; q++)
                if ((D == 3 ? t.kfac_opp[tt][q] : t.tfac_opp[tt][q]) == cs[j]) fj = q;
            const int *fo = D == 3 ? t.kfac_anc[tt][fj] : t.tfac_anc[tt][fj];
            const int ft = D == 3 ? t.kfac_type[tt][fj] : t.tfac_type[tt][fj];
            const int ncof = D == 3 ? t.ntcof[ft] : t.necof[ft];
            int ib = 0;
            for (int i = 0; i < ncof; i++) {
                const int *an = D == 3 ? t.tcof_anc[ft][i] : t.ecof_anc[ft][i];
                const int ty = D == 3 ? t.tcof_type[ft][i] : t.ecof_type[ft][i];
                if (an[0] == -fo[0] && an[1] == -fo[1] && an[2] == -fo[2] && ty == tt) ib = i;
            }
            const int io = 1 - ib;
            const int *an = D == 3 ? t.tcof_anc[ft][io] : t.ecof_anc[ft][io];
            for (int k = 0; k < 3; k++) t.asc_off[tt][j][k] = fo[k] + an[k];
            t.asc_type[tt][j] = D == 3 ? t.tcof_type[ft][io] : t.ecof_type[ft][io];
        }
    }
    for (int tt = 0; tt < T::NT; tt++) {
        const int cs[3] = {0, t.tA[tt], t.tB[tt]};
        for (int j = 0; j < 3; j++)
            for (int q = 0; q < 3; q++)
                if (t.tfac_opp[tt][q] == cs[j]) t.tri_opp[tt][j] = q;
    }
    t.nwin = 0;
    for (int z = zlo; z <= zhi; z++)
        for (int y = -1; y <= 2; y++)
            for (int x = -1; x <= 2; x++) {
                const bool lowcube = x <= 1 && y <= 1 && z <= 1, highcube = x >= 0 && y >= 0 && z >= 0;
                if (!lowcube && !highcube) continue;
                t.win[t.nwin][0] = x; t.win[t.nwin][1] = y; t.win[t.nwin][2] = z;
                t.nwin++;
            }
    // dense evaluator positions
    for (int k = 0; k < T::NC; k++) {
        int cx = k & 1, cy = (k >> 1) & 1, cz = (k >> 2) & 1;
        t.cpos[k] = wpos<D>(cx, cy, cz);
        for (int n = 0; n < T::NNB; n++) t.cnb[k][n] = wpos<D>(cx + t.nb[n][0], cy + t.nb[n][1], cz + t.nb[n][2]);
        for (int n = 0; n < T::NNB; n++) t.cnb_ord[k][n] = n;
        for (int i = 1; i < T::NNB; i++)
            for (int j = i; j > 0 && t.cnb[k][t.cnb_ord[k][j - 1]] > t.cnb[k][t.cnb_ord[k][j]]; j--) {
                int u = t.cnb_ord[k][j]; t.cnb_ord[k][j] = t.cnb_ord[k][j - 1]; t.cnb_ord[k][j - 1] = u;
            }
    }
    {
        int k = 0;
        for (int b = 1; b <= T::AX; b++) { t.ce_a[k] = 0; t.ce_b[k] = b; k++; }
        for (int a = 1; a <= T::AX; a++)
            for (int b = 1; b <= T::AX; b++)
                if ((a & b) == a && a != b) { t.ce_a[k] = a; t.ce_b[k] = b; k++; }
        for (int ce = 0; ce < T::NCE; ce++) {
            int a = t.ce_a[ce], ty = (t.ce_b[ce] ^ a) - 1;
            int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
            t.ce_ncof[ce] = t.necof[ty];
            for (int i = 0; i < t.necof[ty]; i++)
                t.ce_cof[ce][i] = wpos<D>(ax + t.ecof_v[ty][i][0], ay + t.ecof_v[ty][i][1], az + t.ecof_v[ty][i][2]);
        }
    }
    {
        int k = 0;
        for (int tt = 0; tt < T::NT; tt++) { t.ct_a[k] = 0; t.ct_b[k] = t.tA[tt]; t.ct_c[k] = t.tB[tt]; k++; }
        for (int a = 1; a <= T::AX; a++)
            for (int b = 1; b <= T::AX; b++)
                for (int c = 1; c <= T::AX; c++)
                    if ((a & b) == a && a != b && (b & c) == b && b != c) { t.ct_a[k] = a; t.ct_b[k] = b; t.ct_c[k] = c; k++; }
        for (int ct = 0; ct < T::NCT; ct++) {
            const int cs[3] = {t.ct_a[ct], t.ct_b[ct], t.ct_c[ct]};
            const int ends[3][3] = {{0, 1, 2}, {0, 2, 1}, {1, 2, 0}};   // (x, y, opposite)
            for (int j = 0; j < 3; j++) {
                int x = cs[ends[j][0]], y = cs[ends[j][1]], o = cs[ends[j][2]];
                int idx = -1;
                for (int ce = 0; ce < T::NCE; ce++) if (t.ce_a[ce] == x && t.ce_b[ce] == y) idx = ce;
                t.ct_e[ct][j] = idx;
                int op = wpos<D>(o & 1, (o >> 1) & 1, (o >> 2) & 1), pos = -1;
                for (int i = 0; i < t.ce_ncof[idx]; i++) if (t.ce_cof[idx][i] == op) pos = i;
                t.ct_opp_pos[ct][j] = pos;
            }
            int a = cs[0], ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
            int ty = tri_type_of<D>(cs[1] ^ a, cs[2] ^ a);
            t.ct_ncof[ct] = t.ntcof[ty];
            for (int i = 0; i < t.ntcof[ty]; i++)
                t.ct_cof[ct][i] = wpos<D>(ax + t.tcof_v[ty][i][0], ay + t.tcof_v[ty][i][1], az + t.tcof_v[ty][i][2]);
        }
    }
    for (int kk = 0; kk < T::NK; kk++) {
        const int cs[4] = {0, t.kA[kk], t.kB[kk], 7};
        for (int j = 0; j < 4; j++) {
            int rest[3] = {}, m = 0;
            for (int i = 0; i < 4; i++) if (i != j) rest[m++] = cs[i];
            int idx = -1;
            for (int ct = 0; ct < T::NCT; ct++)
                if (t.ct_a[ct] == rest[0] && t.ct_b[ct] == rest[1] && t.ct_c[ct] == rest[2]) idx = ct;
            t.k_tri[kk][j] = idx;
            int o = cs[j], op = wpos<D>(o & 1, (o >> 1) & 1, (o >> 2) & 1), pos = -1;
            for (int i = 0; i < t.ct_ncof[idx]; i++) if (t.ct_cof[idx][i] == op) pos = i;
            t.k_opp_pos[kk][j] = pos;
        }
    }
    return t;
}

// compile-time copy: every access with constant indices folds to an immediate
template <int D> struct TabC {
    static constexpr Tab<D> T = make_tab<D>();
};

// ------------------------------------------------------------------------------------
// code fields
// ------------------------------------------------------------------------------------
template <int D> MSC_HD __forceinline__ int vfield(uint64_t c) { return (int)(c & 15u); }
template <int D> MSC_HD __forceinline__ int efield(uint64_t c, int t) { return (int)((c >> (4 + 3 * t)) & 7u); }
template <int D> MSC_HD __forceinline__ int tfield(uint64_t c, int t)
{
    return (int)((c >> (Tab<D>::TRI_BIT0 + 2 * t)) & 3u);
}
template <int D> MSC_HD __forceinline__ int kfield(uint64_t c, int t)
{
    return (int)((c >> (Tab<D>::TET_BIT0 + t)) & 1u);
}

// SoS order between two window positions known at compile time (i != j)
#define MSC_WLT(w, i, j) ((i) < (j) ? ((w)[i] <= (w)[j]) : ((w)[i] < (w)[j]))

// compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1
template <class F, int... I>
MSC_HD __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F> MSC_HD __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Discrete gradient of every cell owned by one anchor (Sec. 4.2 pairing rules):
//  vertex: pairs with the edge to its lowest lower neighbour;
//  edge ab (a > b): paired down if a's pair is ab; else pairs with triangle abc whose c is
//    the lowest vertex below both a and b; else critical;
//  triangle abc: paired down if its highest edge (opposite its lowest vertex) chose it;
//    else pairs with the tet whose extra vertex is lowest among those below a, b, c;
//  tetrahedron: paired down if its highest triangle chose it; else critical (a maximum).
// w: the WS window values (+inf outside the domain); corner_in: bit k set if cube corner
// k of the anchor lies in the domain.  Every table index is a compile-time constant.
// Each "lowest candidate below X" is found as the SoS-lowest candidate overall (candidates
// visited by increasing vertex id, replaced only by a strictly smaller value) followed by
// one comparison with X: the overall lowest is below X exactly when any candidate is.
template <int D>
MSC_HD __forceinline__ uint64_t eval_anchor(const float *w, unsigned corner_in)
{
    using Tb = Tab<D>;
    int vp[Tb::NC];
    static_for<Tb::NC>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int ck = TabC<D>::T.cpos[k];
        float bv = pos_inf();
        int bn = 15;
        static_for<Tb::NNB>([&](auto ic) {
            constexpr int n = TabC<D>::T.cnb_ord[k][decltype(ic)::value];
            constexpr int q = TabC<D>::T.cnb[k][n];
            if (w[q] < bv) { bv = w[q]; bn = n; }
        });
        // a neighbour -e_A (index >= NE) has the smaller vertex id, so it wins a tie
        const bool below = bv < w[ck] || (bv == w[ck] && bn >= Tb::NE);
        vp[k] = below ? bn : 15;
    });
    int eup[Tb::NCE];   // -2 paired down, -1 critical, >= 0 index of the cofacet taken
    static_for<Tb::NCE>([&](auto cc) {
        constexpr int ce = decltype(cc)::value;
        constexpr int a = TabC<D>::T.ce_a[ce], b = TabC<D>::T.ce_b[ce];
        constexpr int pa = TabC<D>::T.cpos[a], pb = TabC<D>::T.cpos[b];
        constexpr int d = (b ^ a) - 1;
        const bool a_hi = MSC_WLT(w, pb, pa);
        const bool down = a_hi ? (vp[a] == d) : (vp[b] == Tb::NE + d);
        float bv = pos_inf();
        int bp = 1 << 20, bi = -1;
        static_for<TabC<D>::T.ce_ncof[ce]>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int q = TabC<D>::T.ce_cof[ce][i];
            if (w[q] < bv) { bv = w[q]; bp = q; bi = i; }
        });
        const bool below = (bv < w[pa] || (bv == w[pa] && bp < pa)) && (bv < w[pb] || (bv == w[pb] && bp < pb));
        eup[ce] = down ? -2 : (below ? bi : -1);
    });
    int tup[Tb::NCT];   // -2 paired down, -1 critical, >= 0 index of the cofacet tet taken
    static_for<Tb::NCT>([&](auto tc) {
        constexpr int ct = decltype(tc)::value;
        constexpr int pa = TabC<D>::T.cpos[TabC<D>::T.ct_a[ct]];
        constexpr int pb = TabC<D>::T.cpos[TabC<D>::T.ct_b[ct]];
        constexpr int pc = TabC<D>::T.cpos[TabC<D>::T.ct_c[ct]];
        const bool la = MSC_WLT(w, pa, pb) && MSC_WLT(w, pa, pc);
        const bool lb = !la && MSC_WLT(w, pb, pc);
        // the highest edge is opposite the lowest vertex: (b,c) if a is lowest, (a,c) if b, (a,b) if c
        constexpr int e0 = TabC<D>::T.ct_e[ct][0], e1 = TabC<D>::T.ct_e[ct][1], e2 = TabC<D>::T.ct_e[ct][2];
        constexpr int o0 = TabC<D>::T.ct_opp_pos[ct][0], o1 = TabC<D>::T.ct_opp_pos[ct][1];
        constexpr int o2 = TabC<D>::T.ct_opp_pos[ct][2];
        const int hi_up = la ? eup[e2] : (lb ? eup[e1] : eup[e0]);
        const int want = la ? o2 : (lb ? o1 : o0);
        const bool down = hi_up == want;
        float bv = pos_inf();
        int bp = 1 << 20, bi = -1;
        static_for<TabC<D>::T.ct_ncof[ct]>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int q = TabC<D>::T.ct_cof[ct][i];
            if (w[q] < bv) { bv = w[q]; bp = q; bi = i; }
        });
        // below all three vertices = below the lowest one
        const float lv = la ? w[pa] : (lb ? w[pb] : w[pc]);
        const int lp = la ? pa : (lb ? pb : pc);
        const bool below = bv < lv || (bv == lv && bp < lp);
        tup[ct] = down ? -2 : (below ? bi : -1);
    });
    uint64_t code = (uint64_t)vp[0];
    static_for<Tb::NE>([&](auto ec) {
        constexpr int e = decltype(ec)::value;
        const int f = eup[e] == -2 ? 1 : (eup[e] >= 0 ? 2 + eup[e] : 0);
        if ((corner_in >> (e + 1)) & 1u) code |= (uint64_t)f << (4 + 3 * e);
    });
    static_for<Tb::NT>([&](auto tc) {
        constexpr int t = decltype(tc)::value;
        const int f = tup[t] == -2 ? 1 : (tup[t] >= 0 ? 2 + tup[t] : 0);
        constexpr int top = TabC<D>::T.tB[t];
        if ((corner_in >> top) & 1u) code |= (uint64_t)f << (Tb::TRI_BIT0 + 2 * t);
    });
    static_for<Tb::NK>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int c0 = TabC<D>::T.cpos[0], c1 = TabC<D>::T.cpos[TabC<D>::T.kA[k]];
        constexpr int c2 = TabC<D>::T.cpos[TabC<D>::T.kB[k]], c3 = TabC<D>::T.cpos[7];
        const bool l0 = MSC_WLT(w, c0, c1) && MSC_WLT(w, c0, c2) && MSC_WLT(w, c0, c3);
        const bool l1 = !l0 && MSC_WLT(w, c1, c2) && MSC_WLT(w, c1, c3);
        const bool l2 = !l0 && !l1 && MSC_WLT(w, c2, c3);
        // the highest facet is the one opposite the lowest corner
        constexpr int t0 = TabC<D>::T.k_tri[k][0], t1 = TabC<D>::T.k_tri[k][1];
        constexpr int t2 = TabC<D>::T.k_tri[k][2], t3 = TabC<D>::T.k_tri[k][3];
        constexpr int q0 = TabC<D>::T.k_opp_pos[k][0], q1 = TabC<D>::T.k_opp_pos[k][1];
        constexpr int q2 = TabC<D>::T.k_opp_pos[k][2], q3 = TabC<D>::T.k_opp_pos[k][3];
        const int down = l0 ? (tup[t0] == q0) : l1 ? (tup[t1] == q1) : l2 ? (tup[t2] == q2) : (tup[t3] == q3);
        if ((corner_in >> 7) & 1u) code |= (uint64_t)down << (Tb::TET_BIT0 + k);
    });
    return code;
}

}  // namespace msc
