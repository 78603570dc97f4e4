// stream_layout.h -- byte layout of a level-program stream (host builder and device
// consumer share these formulas).
//
// A program for one subdomain is a run of fixed-size chunks (one TMA bulk copy fills one
// shared-memory ring stage with one chunk). A chunk holds
//   a 16-byte header {uint32 nseg},
//   a segment table of nseg 8-byte entries (padded to 16 bytes):
//       word 0: bits 0..15  offset of the segment's first record, in 16-byte units
//               bits 16..24 width: records per wave (<= the consumer group's threads)
//       word 1: bits 0..15  waves in the segment
//               bit  29     synchronise the consumer group after every wave (a run of
//                           levels, one wave each)
//               bit  30     a scan segment (below)
//               bit  31     synchronise the consumer group after the segment
//   the records of every segment, wave after wave, each wave `width` records.
// Consumer thread t runs record t of every wave of a segment, in wave order; threads
// synchronise only where a segment carries the barrier bit. Within the rows between two
// barriers no thread reads or overwrites a slot another thread writes or reads there
// (the builder arranges this; a thread's own program order covers everything else).
//
// Scan segments (width a multiple of 32) hold chains: warp u takes records 32u..32u+31 of
// each wave, and the records a warp takes, wave after wave, form its sequence. A record
// may be linked to the one before it in the sequence: it reads that row's result through
// its first column (head bit 30) or in its own slot (head bit 29). A wave's 32 rows are
// then x_l = a_l + b_l x_{l-1}, a_l and b_l formed from values final before the wave, and
// the warp composes the affine maps by a prefix scan over its lanes; lane 0 reads its
// predecessor (stored by the previous wave) from the vector. Every other value a record
// reads was final before its segment or written by its own warp in an earlier wave; scan
// stretches hold scan segments only and end at a barrier.
//
// A row record (16-byte aligned, read with 128-bit shared-memory loads) holds
//   uint32 head      element index of x[row] | (n << 24) | link bits 29, 30; bit 31 marks a
//                    skip record
//   T      dinv      1 / u_ii for an upper-triangular row, 1 for a unit-lower row
//   uint32 col[RW]   byte offsets of x[col]; entries n.. hold the row's own offset
//   V      val[RW]   entries n.. hold zero (V = T, or bfloat16 with T = float)
// and computes x[row] = (x[row] - sum_{q<RW} val[q] * x[col[q]]) * dinv, the sum formed
// pairwise. The padded entries add exact zeros, so every record takes the same
// branch-free path. A skip record (a hole in a wave) reads slot 0 and stores nothing.
// Column offsets are pre-scaled by the element size so the consumer adds them to the
// vector's base; the row index is scaled on use (24 bits: up to 2^24 rows per subdomain in
// either precision).
#pragma once

#include <stdint.h>

namespace ilu2l {

constexpr int kChunkHdr = 16;
constexpr int kSegEntry = 8;
constexpr uint32_t kSegBarrier = 1u << 31;
constexpr uint32_t kSegScan = 1u << 30;
constexpr uint32_t kSegSyncEach = 1u << 29;
constexpr uint32_t kRecLinkCol = 1u << 30;   // linked through col[0]
constexpr uint32_t kRecLinkSelf = 1u << 29;  // linked through the own slot
constexpr uint32_t kRecNMask = 0x1Fu;        // (head >> 24) & kRecNMask = n (<= 16)
constexpr uint32_t kSegMaxWaves = 0xFFFF;
constexpr uint32_t kRecSkip = 1u << 31;
// consumer threads of a stream kernel (its block has 256: one more warp hosts the
// thread that refills the ring)
constexpr int kMaxConsumers = 224;

#ifdef __CUDACC__
#define ILU2L_HD __host__ __device__ __forceinline__
#else
#define ILU2L_HD inline
#endif

ILU2L_HD constexpr uint32_t al(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

struct RecLayout {
    uint32_t dinv, col, val, bytes;
};

// byte offsets of dinv, col and val and the record size, for values of val_bytes and
// vector elements (and dinv) of x_bytes
ILU2L_HD constexpr RecLayout rec_layout(uint32_t rw, uint32_t val_bytes, uint32_t x_bytes) {
    return RecLayout{x_bytes, 2 * x_bytes, al(2 * x_bytes + rw * 4, val_bytes),
                     al(al(2 * x_bytes + rw * 4, val_bytes) + rw * val_bytes, 16)};
}

}  // namespace ilu2l
