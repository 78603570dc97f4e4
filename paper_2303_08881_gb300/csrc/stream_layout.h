// stream_layout.h -- byte layout of a level-program stream (host builder and device
// consumer share these formulas).
//
// A program for one subdomain is a run of fixed-size chunks (one TMA bulk copy fills one
// shared-memory ring stage with one chunk). A chunk holds
//   a 16-byte header {uint32 nwaves},
//   a wave table of nwaves uint32 entries (padded to 16 bytes):
//       bits 0..15  offset of the wave's first record, in 16-byte units from the chunk
//       bits 16..24 width: records in the wave (<= the consumer group's thread count)
//       bit  25     synchronise the consumer group after this wave (end of a level)
//   the row records of every wave, contiguous per wave.
// A wave holds rows of ONE level, at most one per consumer thread; a level wider than
// the group spans several consecutive waves and only its last wave carries the bit.
//
// A row record (16-byte aligned, read with 128-bit shared-memory loads) holds
//   uint32 head      byte offset of x[row] in the working vector | (n << 24), n <= RW
//   T      dinv      1 / u_ii for an upper-triangular row, 1 for a unit-lower row
//   uint32 col[RW]   byte offsets of x[col] (entries n.. unused)
//   T      val[RW]
// and computes x[row] = (x[row] - sum_{q<n} val[q] * x[col[q]]) * dinv. Offsets are
// pre-scaled by the element size so the consumer adds them to the vector's base.
#pragma once

#include <stdint.h>

namespace ilu2l {

constexpr uint32_t kWaveSync = 1u << 25;
constexpr int kChunkHdr = 16;


#ifdef __CUDACC__
#define ILU2L_HD __host__ __device__ __forceinline__
#else
#define ILU2L_HD inline
#endif

ILU2L_HD constexpr uint32_t al(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

struct RecLayout {
    uint32_t dinv, col, val, bytes;
};

ILU2L_HD constexpr RecLayout rec_layout(uint32_t rw, uint32_t val_bytes) {
    return RecLayout{val_bytes, 2 * val_bytes, al(2 * val_bytes + rw * 4, val_bytes),
                     al(al(2 * val_bytes + rw * 4, val_bytes) + rw * val_bytes, 16)};
}

}  // namespace ilu2l
