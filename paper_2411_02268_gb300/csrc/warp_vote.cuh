// Warp ranking by votes (the radix scatter).
#pragma once

namespace cdk {

// Lanes of the warp whose 8-bit value (low byte of v) equals this lane's,
// among the lanes with ok set (the others form a group of their own): nine
// votes, one per bit and one for ok, instead of a match instruction (whose
// latency stalled the radix scatter; in the bucket scatter, with its block
// barriers between rounds, the match measured faster and stays).  Every lane
// of the warp must call it.
__device__ __forceinline__ unsigned byte_peers(bool ok, unsigned v) {
    const unsigned code = ok ? (v & 255u) : 0x100u;
    unsigned peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        const unsigned bal = __ballot_sync(0xffffffffu, (code >> b) & 1u);
        peers &= ((code >> b) & 1u) ? bal : ~bal;
    }
    return peers;
}

}  // namespace cdk
