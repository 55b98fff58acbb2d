// Size buckets of the mixed-precision forward: which engine takes a row of order m.
// Written by paper_1710_10899_gb300/tune.py from forward times measured on a GB300 (the
// measurements are listed below); rows of order m <= kTunedSmallMaxM go to the small engine
// (working set in shared memory, 16 x 8 warp tiles of mma.sync), rows with
// kTunedSmallMaxM < m <= kTunedSyncMaxM to the mma.sync engine (64 x 64 tiles, cp.async
// pipeline), the rest to the tcgen05 engine (128 x 96 tiles in TMEM, TMA pipeline).
// Device: NVIDIA GB300; p = 2; 7296 rows of one order per case; ms per forward
// (median):
//     m        small      sync   tcgen05
//     8        1.904     6.145     4.508
//    16        2.047     6.788     4.716
//    24        2.291     7.345     5.517
//    32        2.380     7.573     5.630
//    48            -     8.371     6.596
//    64            -     8.975     7.806
//    96            -    25.950    11.104
//   128            -    27.932    15.184
#pragma once
namespace submat {
constexpr int kTunedSmallMaxM = 32;
constexpr int kTunedSyncMaxM = 0;
}  // namespace submat
