// Host build of the CUDA path's per-anchor gradient evaluator (eval_anchor, with its
// compile-time cell tables) and pair decoder, for the CPU test that compares them with the
// oracle: test infrastructure, not part of the library.
#define MSC_HOST_EMULATION 1
#include <cstdint>
#include <vector>

#include "../../paper_2409_17346_gb300/csrc/msc_core.cuh"

template <int D>
static void pairs_of(const float *field, const msc::Grid &G, int64_t *rows, uint64_t cap, uint64_t *n_out)
{
    std::vector<uint64_t> code(G.n);
    for (uint32_t p = 0; p < G.n; p++) code[p] = msc::anchor_code<D>(field, G, p);
    unsigned long long count = 0;
    for (uint32_t p = 0; p < G.n; p++) msc::decode_pairs<D>(code.data(), G, p, rows, &count, cap);
    *n_out = count;
}

// the gradient pairs (L, U) of a field as rows of 8 vertex ids (unsorted), as the library
// reports them; rows may be null to count
extern "C" int host_gradient_pairs(const float *field, int nx, int ny, int nz, int64_t *rows, uint64_t cap,
                                   uint64_t *n_out)
{
    const msc::Grid G = msc::make_grid(nx, ny, nz);
    if (nz > 1) pairs_of<3>(field, G, rows, cap, n_out);
    else pairs_of<2>(field, G, rows, cap, n_out);
    return 0;
}
