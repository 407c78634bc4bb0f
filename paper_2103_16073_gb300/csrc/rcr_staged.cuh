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
// [0, nmax) of pass 0 (rotation) or 1 (back-rotation; K limited by p_in).
void fb_stc_group_tiles(int g, int g0, int g1, int nmax, int pass, int p_in, std::vector<StcTile>& out);

// A tile of the tensor-core coaxial pass: virtual columns [vc0, vc0 + nvc)
// (nvc <= 128; order 0: one slot each, order am > 0: slot (v / 2), even part
// for even v and odd part for odd v) of one |t| set whose slots start at
// cidx[c0], output degrees am + r0 .. am + r0 + nr - 1 (nr <= 128), summed
// over the K = p_in - am input degrees; its pre-split coaxial block starts at
// float toff of the plan's coaxial tables.
struct StcCTile {
    int64_t toff;
    int32_t c0, vc0, nvc;
    int32_t am, r0, nr, K;
    int32_t pad;
};
// A pre-split coaxial block to build: C^{am}_{am + r0 + i, am + k} of the set
// at coax offset cs_off (row stride pc), i < nr, k < K, at float toff.
struct StcCBlock {
    int64_t cs_off, toff;
    int32_t pc, am, r0, nr, K, pad;
};
constexpr int STC_CROWS = 128;   // coaxial output rows (complex) per tile

// Appends the coaxial tiles and table blocks of one |t| set (ns slots at
// cidx[c0], coefficients at cs_off, stride pc) of a level; *tfloats grows by
// the floats of the new table blocks.
void fb_stc_coax_set(int c0, int ns, int64_t cs_off, int pc, int p_in, int p_out, std::vector<StcCTile>& tiles,
                     std::vector<StcCBlock>& blocks, int64_t* tfloats);
// Builds the pre-split coaxial blocks (3xTF32 real form of the complex
// blocks) from the FP64 coaxial sets.
fb_status fb_stc_coax_tables(const StcCBlock* blocks, int nblocks, const cd* coax64, float* out, cudaStream_t s);
// Launches the coaxial tiles: U -> V (both degree-major folded).
fb_status fb_stc_coax_run(const StcCTile* tiles, int ntiles, const int32_t* cidx, const float* tab, const cf* U,
                          cf* V, int S, int p_out, int* err, cudaStream_t s);

// Launches the rotation (pass 0) or back-rotation (pass 1) tiles.
fb_status fb_stc_run(int pass, const StcTile* tiles, int ntiles, int npmax, const int64_t* toff, const float* tab,
                     int64_t tper, const StgSlot* slots, const cf* X, cf* out, int S, int p_in, int p_out,
                     const cf* rph, int prot, int* err, cudaStream_t s);

}  // namespace stg
