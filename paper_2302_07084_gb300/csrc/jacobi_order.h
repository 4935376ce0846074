// Pairing order of the register-resident one-sided Jacobi (dense.cu,
// jacobi_reg_kernel): the index arithmetic only, shared by the kernel and by
// a host-side check of the order.
//
// m = 2G columns sit in G groups of two slots. A sweep:
//  - level 0: the slot-0 columns form a set X, the slot-1 columns a set Y;
//    for r = 0..G-1 group i pairs X[i] with Y[(i + r) mod G], so between
//    rounds only the slot-1 column moves, from group i + 1 (cyclically);
//  - level l > 0: every set of the level before is split into its halves
//    (one move of both slots, jorder_split_sources), and the same ring runs
//    inside each half, in parallel; this continues while the set size is
//    even;
//  - sets of odd size s >= 3 then finish with s rounds of the circle method
//    (jorder_tail_sources): ring positions 1..k of a set are paired with
//    s-1..k+1 in k groups, position 0 is idle, and the two sets that share a
//    parent put their idle columns in one group.
// Sources are entries group * 2 + slot of the layout before the move. Every
// pair of columns meets exactly once per sweep, and the layout a sweep ends
// with is the next sweep's starting layout.
#pragma once

#ifdef __CUDACC__
#define LNE_JORDER_FN __host__ __device__ __forceinline__
#else
#define LNE_JORDER_FN inline
#endif

namespace lne {

// number of halving levels: the trailing zero bits of m (m even, > 0)
LNE_JORDER_FN int jorder_levels(int m) {
    int tz = 0;
    while (((m >> tz) & 1) == 0) ++tz;
    return tz;
}

// rounds per sweep
LNE_JORDER_FN int jorder_rounds(int m) { return (m >> jorder_levels(m)) > 1 ? m : m - 1; }

// ring move inside a set of h groups: the group whose slot-1 column group g takes
LNE_JORDER_FN int jorder_ring_source(int g, int h) {
    const int j = g / h, i = g - j * h;
    return j * h + (i + 1 == h ? 0 : i + 1);
}

// entering a level whose ring length is h: each set of 2h groups of the level
// before (ending at its last ring round) becomes two sets of h groups
LNE_JORDER_FN void jorder_split_sources(int g, int h, int &src0, int &src1) {
    const int H = 2 * h, jp = g / H, x = g - jp * H, half = x >= h ? 1 : 0, ip = x - half * h;
    src0 = half ? (jp * H + (ip + 1) % H) * 2 + 1 : (jp * H + ip) * 2;
    src1 = half ? (jp * H + (h + ip + 1) % H) * 2 + 1 : (jp * H + h + ip) * 2;
}

// odd-set rounds (set size s >= 3): sources entering them from the last ring
// round (e0, e1) and between two of them (r0, r1); idle: this group pairs two
// idle columns and does not rotate
LNE_JORDER_FN void jorder_tail_sources(int g, int s, int &e0, int &e1, int &r0, int &r1, bool &idle) {
    const int k = (s - 1) / 2, base = (g / s) * s, x = g - base;
    idle = x == s - 1;
    const int sub0 = idle ? 0 : x / k, p0 = idle ? 0 : x - sub0 * k + 1;
    const int sub1 = idle ? 1 : sub0, p1 = idle ? 0 : s - p0;
    // (group, slot) of ring position p of set sb (0: first half of the parent, 1: second)
    auto posmap = [&](int sb, int p) {
        return p == 0 ? (base + s - 1) * 2 + sb
                      : p <= k ? (base + sb * k + p - 1) * 2 : (base + sb * k + (s - p) - 1) * 2 + 1;
    };
    // member y of a set at the end of the last ring level
    auto ring_end = [&](int sb, int y) { return sb == 0 ? (base + y) * 2 : (base + (y + 1) % s) * 2 + 1; };
    e0 = ring_end(sub0, p0);
    e1 = ring_end(sub1, p1);
    r0 = posmap(sub0, (p0 + 1) % s);
    r1 = posmap(sub1, (p1 + 1) % s);
}

}  // namespace lne

#undef LNE_JORDER_FN
