// Layouts shared by the staged RCR passes on CUDA cores (rcr_staged.cu) and
// their tensor-core rotation passes (rcr_staged_tc.cu).
#pragma once

#include <cstdint>
#include <vector>

#include "common.cuh"

namespace stg {

// one pair (column) of a staged level
struct StgSlot {
    int64_t src_off;   // first coefficient of the source expansion
    int64_t dst_off;   // first coefficient of the target expansion
    int32_t dir;       // translation direction (phase table)
    int32_t pad;
};

// start of degree n in the unfolded rotation factors of one direction
__host__ __device__ __forceinline__ int64_t rot_off(int n) { return (int64_t)n * (2 * n - 1) * (2 * n + 1) / 3; }

// start of order m in the order-major layout of an order-p expansion
// (orders -(p-1) .. p-1, order m holding degrees |m| .. p-1)
__host__ __device__ __forceinline__ int moff(int m, int p) {
    if (m <= 0) {
        int a = p + m;   // p - |m|
        return (a - 1) * a / 2;
    }
    return (p - 1) * p / 2 + m * p - m * (m - 1) / 2;
}

// start of degree n in a folded rotation table (blocks (n+1)^2 + n^2)
__host__ __device__ __forceinline__ int64_t fo(int n) {
    return (int64_t)(n - 1) * n * (2 * n - 1) / 3 + (int64_t)n * n;
}

// ---- tensor-core rotation passes ------------------------------------------
// A tile of the tensor-core R or B pass: slots [s0, s0 + ns) (ns <= 64) of
// one polar-angle group g, folded part `part`, degrees [n0, n1), whose
// accumulators share the CTA's tensor memory.
struct StcTile {
    int32_t g, part;
    int32_t n0, n1;
    int32_t s0, ns;
};

constexpr int STC_SLOTS = 64;        // slots per tile (128 real rows: re, im)
constexpr int STC_TMEM_COLS = 256;   // accumulator columns per tile

// columns of the folded degree-n block (rows of the table), padded to 16
__host__ __device__ __forceinline__ int stc_pad16(int v) { return (v + 15) & ~15; }

// Float offsets of the pre-split canonical table blocks of one group and
// pass: toff[2 n + part] for degrees n < P (square blocks of
// stc_pad16(n + 1 - part) rows and K values, K chunks of 16 each holding the
// TF32 part then the remainder); returns the floats per group and pass.
int64_t fb_stc_layout(int P, std::vector<int64_t>& toff);

// Appends the tiles of one polar-angle group (slots [g0, g1)) for degrees
// [0, nmax) of a pass; kdeg(n) = K of degree n (0: no block).
void fb_stc_group_tiles(int g, int g0, int g1, int nmax, int pass, int p_in, std::vector<StcTile>& out);

// Launches the rotation (pass 0) or back-rotation (pass 1) tiles.
fb_status fb_stc_run(int pass, const StcTile* tiles, int ntiles, int npmax, const int64_t* toff, const float* tab,
                     int64_t tper, const StgSlot* slots, const cf* X, cf* out, int S, int p_in, int p_out,
                     const cf* rph, int prot, int* err, cudaStream_t s);

}  // namespace stg
