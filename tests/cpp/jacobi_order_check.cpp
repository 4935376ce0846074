// Host check of the register-resident Jacobi's pairing order
// (paper_2302_07084_gb300/csrc/jacobi_order.h, the same functions the kernel
// calls): for every column count c = 1..160 and three consecutive sweeps,
// every move is a permutation of the (group, slot) entries with sources in
// range, every pair of columns meets exactly once per sweep (pairs in idle
// groups excluded), and a sweep has jorder_rounds(m) rounds.
#include <cstdio>
#include <vector>

#include "jacobi_order.h"

using namespace lne;

int main() {
    int failures = 0;
    for (int c = 1; c <= 160; ++c) {
        const int m = c + (c & 1), G = m / 2;
        std::vector<int> lay(2 * G);   // lay[g * 2 + slot] = column held there
        for (int g = 0; g < G; ++g) {
            lay[2 * g] = g;
            lay[2 * g + 1] = g + G;
        }
        for (int sweep = 0; sweep < 3; ++sweep) {
            bool ok = true;
            std::vector<char> met((size_t)m * m, 0);
            int rounds = 0, pairs = 0;
            auto move = [&](const std::vector<int> &src) {   // src[g * 2 + slot]
                std::vector<char> used(2 * G, 0);
                std::vector<int> nl(2 * G);
                for (int e = 0; e < 2 * G; ++e) {
                    const int s = src[e];
                    if (s < 0 || s >= 2 * G || used[s]) {
                        ok = false;
                        return;
                    }
                    used[s] = 1;
                    nl[e] = lay[s];
                }
                lay = nl;
            };
            auto pair_round = [&](const std::vector<char> &active) {
                ++rounds;
                for (int g = 0; g < G; ++g) {
                    if (!active[g]) continue;
                    const int a = lay[2 * g], b = lay[2 * g + 1];
                    if (a == b || met[(size_t)a * m + b]) ok = false;
                    met[(size_t)a * m + b] = met[(size_t)b * m + a] = 1;
                    ++pairs;
                }
            };
            const std::vector<char> all(G, 1);
            const int L = jorder_levels(m), s = m >> L;
            for (int lev = 0; lev < L; ++lev) {
                const int h = m >> (lev + 1);
                if (lev > 0) {
                    std::vector<int> src(2 * G);
                    for (int g = 0; g < G; ++g) jorder_split_sources(g, h, src[2 * g], src[2 * g + 1]);
                    move(src);
                }
                for (int r = 0; r < h; ++r) {
                    if (r > 0) {
                        std::vector<int> src(2 * G);
                        for (int g = 0; g < G; ++g) {
                            src[2 * g] = 2 * g;
                            src[2 * g + 1] = 2 * jorder_ring_source(g, h) + 1;
                        }
                        move(src);
                    }
                    pair_round(all);
                }
            }
            if (s > 1) {
                std::vector<int> e(2 * G), rr(2 * G);
                std::vector<char> active(G);
                for (int g = 0; g < G; ++g) {
                    bool idle = false;
                    jorder_tail_sources(g, s, e[2 * g], e[2 * g + 1], rr[2 * g], rr[2 * g + 1], idle);
                    active[g] = !idle;
                }
                for (int r = 0; r < s; ++r) {
                    move(r == 0 ? e : rr);
                    pair_round(active);
                }
            }
            if (rounds != jorder_rounds(m) || pairs != m * (m - 1) / 2) ok = false;
            if (!ok) {
                std::printf("c = %d, sweep %d: invalid order (rounds %d, pairs %d)\n", c, sweep, rounds, pairs);
                ++failures;
                break;
            }
        }
    }
    std::printf(failures ? "FAIL\n" : "ok\n");
    return failures ? 1 : 0;
}
