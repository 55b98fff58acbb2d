// Size buckets of the mixed-precision forward: which engine takes a row of order m.
// Written by paper_1710_10899_gb300/tune.py from forward times measured on a GB300 (the
// measurements are listed below); rows of order m <= kTunedSmallMaxM go to the small engine
// (working set in shared memory, 16 x 8 warp tiles of mma.sync), rows with
// kTunedSmallMaxM < m <= kTunedSyncMaxM to the mma.sync engine (64 x 64 tiles, cp.async
// pipeline), the rest to the tcgen05 engine (128 x 96 tiles in TMEM, TMA pipeline).
// Device: NVIDIA GB300; p = 2; 7296 rows of one order per case; ms per forward
// (median):
//     m        small      sync   tcgen05
//     8        1.897     6.596     4.485
//    16        2.073     7.461     4.742
//    24        2.391     8.194     5.705
//    32        2.509     8.407     5.951
//    48            -     9.307     7.140
//    64            -     9.939     8.151
//    96            -    31.192    11.897
//   128            -    33.562    16.978
#pragma once
namespace submat {
constexpr int kTunedSmallMaxM = 32;
constexpr int kTunedSyncMaxM = 0;
}  // namespace submat
