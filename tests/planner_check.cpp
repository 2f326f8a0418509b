// Host-side checks of the fusion planner (paper_1612_08091_gb300/csrc/planner.cpp),
// built and run by tests/test_planner_cpu.py without a GPU.
//
//  1. block_matrix: the fused block of random gates (dense on 1-3 targets,
//     X, diagonal, with and without controls) equals the ordered product of
//     the gates embedded element by element, computed here independently.
//  2. plan_greedy on random circuits: every gate is executed exactly once;
//     gates sharing a qubit keep their program order; a dense block spans at
//     most kmax qubits and contains its members' qubits; a diagonal block
//     holds only diagonal gates and its table is the diagonal of the product;
//     plan_greedy_each hands out the same items as plan_greedy.
//  3. permutation blocks on permutation-heavy random circuits (X with 0-2
//     controls, SWAP, some dense and diagonal gates): every gate once, in
//     program order on every qubit; a permutation block holds only
//     permutation gates on at most 12 qubits, is at least perm_min wide, and
//     its table is the permutation of the embedded matrix product.
//  4. product items on circuits of one-qubit layers (H and X on each wire,
//     sometimes a general gate) between wide multi-controlled gates: every
//     gate once, in program order on every qubit; a product item holds only
//     uncontrolled one-qubit gates on at least prod_min qubits, each of its
//     wires continues with a gate wider than kmax (or ends), its matrix of
//     each wire is the ordered product of that wire's member gates and is
//     c times a +-1 matrix with orthogonal rows (M M^T = 2 c^2 I).
//  5. the 30-qubit QFT: the phase gates between two groups of 6 qubits go
//     into one 12-qubit diagonal block (36 gates), 20 items in all.
#include <algorithm>
#include <cstdio>
#include <random>

#include "../paper_1612_08091_gb300/csrc/internal.h"

namespace {

std::mt19937_64 rng(1612);
std::uniform_real_distribution<double> unif(-1.0, 1.0);

// kind 0 dense (1..3 targets), 1 X, 2 diagonal; targets and controls drawn from pool
GateRec random_gate(const std::vector<int> &pool, int kind) {
    std::vector<int> perm = pool;
    std::shuffle(perm.begin(), perm.end(), rng);
    GateRec g;
    const int k = (int)pool.size();
    g.t = kind == 0 ? 1 + (int)(rng() % (uint64_t)std::min(3, k)) : 1;
    const int nc = std::min<int>((int)(rng() % 3), k - g.t);
    for (int j = 0; j < g.t; ++j) {
        g.targets[j] = perm[j];
        g.tmask |= 1ull << perm[j];
    }
    for (int j = 0; j < nc; ++j) {
        g.controls.push_back(perm[g.t + j]);
        g.cmask |= 1ull << perm[g.t + j];
    }
    const int T = 1 << g.t;
    g.m.assign((size_t)T * T, cd(0.0, 0.0));
    if (kind == 1) {
        g.kind = GK_X;
        g.m[1] = g.m[2] = 1.0;
    } else if (kind == 2) {
        g.kind = GK_DIAG1;
        g.diag = true;
        for (int r = 0; r < T; ++r) g.m[(size_t)r * T + r] = std::polar(1.0, 3.0 * unif(rng));
    } else {
        g.kind = GK_DENSE;
        for (auto &z : g.m) z = cd(unif(rng), unif(rng));
    }
    g.perm = perm_map(g, g.pmap);
    return g;
}

// SWAP of two qubits of the pool as a 2-target permutation matrix
GateRec swap_gate(const std::vector<int> &pool) {
    std::vector<int> perm = pool;
    std::shuffle(perm.begin(), perm.end(), rng);
    GateRec g;
    g.t = 2;
    g.targets[0] = perm[0];
    g.targets[1] = perm[1];
    g.tmask = (1ull << perm[0]) | (1ull << perm[1]);
    g.m.assign(16, cd(0.0, 0.0));
    g.m[0 * 4 + 0] = g.m[1 * 4 + 2] = g.m[2 * 4 + 1] = g.m[3 * 4 + 3] = 1.0;
    g.kind = GK_DENSE;
    g.perm = perm_map(g, g.pmap);
    return g;
}

// the gate as a D x D matrix on the block qubits S (bit j of an index = S[j])
std::vector<cd> embed(const GateRec &g, const std::vector<int> &S) {
    const int k = (int)S.size(), D = 1 << k, T = 1 << g.t;
    auto bit = [&](int x, int qubit) {
        for (int j = 0; j < k; ++j)
            if (S[j] == qubit) return (x >> j) & 1;
        return -1;
    };
    std::vector<cd> G((size_t)D * D, cd(0.0, 0.0));
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            bool same = true;  // bits outside the targets agree
            for (int j = 0; j < k; ++j) {
                bool target = false;
                for (int t = 0; t < g.t; ++t) target |= g.targets[t] == S[j];
                if (!target && ((r >> j) & 1) != ((c >> j) & 1)) same = false;
            }
            if (!same) continue;
            bool on = true;
            for (int cq : g.controls) on = on && bit(c, cq) == 1;
            if (!on) {
                G[(size_t)r * D + c] = r == c ? 1.0 : 0.0;
                continue;
            }
            int ri = 0, ci = 0;
            for (int t = 0; t < g.t; ++t) {
                ri |= bit(r, g.targets[t]) << t;
                ci |= bit(c, g.targets[t]) << t;
            }
            G[(size_t)r * D + c] = g.m[(size_t)ri * T + ci];
        }
    return G;
}

std::vector<cd> matmul(const std::vector<cd> &A, const std::vector<cd> &B, int D) {
    std::vector<cd> C((size_t)D * D, cd(0.0, 0.0));
    for (int r = 0; r < D; ++r)
        for (int m = 0; m < D; ++m)
            for (int c = 0; c < D; ++c) C[(size_t)r * D + c] += A[(size_t)r * D + m] * B[(size_t)m * D + c];
    return C;
}

int check_block_matrix() {
    double worst = 0.0;
    for (int trial = 0; trial < 300; ++trial) {
        const int k = 2 + trial % 5, n = 10;
        std::vector<int> all(n);
        for (int i = 0; i < n; ++i) all[i] = i;
        std::shuffle(all.begin(), all.end(), rng);
        std::vector<int> S(all.begin(), all.begin() + k);
        std::sort(S.begin(), S.end());
        const int D = 1 << k;
        std::vector<GateRec> q;
        PlanItem it;
        it.fused = true;
        it.k = k;
        for (int j = 0; j < k; ++j) it.qubits[j] = S[j];
        std::vector<cd> ref((size_t)D * D, cd(0.0, 0.0));
        for (int i = 0; i < D; ++i) ref[(size_t)i * D + i] = 1.0;
        for (int gi = 0; gi < 6; ++gi) {
            q.push_back(random_gate(S, (int)(rng() % 3)));
            it.members.push_back(gi);
            ref = matmul(embed(q.back(), S), ref, D);
        }
        block_matrix(q, it);
        for (size_t i = 0; i < ref.size(); ++i) worst = std::max(worst, std::abs(it.m[i] - ref[i]));
    }
    printf("block_matrix: max |difference| %.3e over 300 blocks\n", worst);
    return worst < 1e-12 ? 0 : 1;
}

int check_plans() {
    int bad = 0;
    for (int trial = 0; trial < 60; ++trial) {
        const int n = 8 + trial % 9, kmax = 2 + trial % 5, G = 40 + (int)(rng() % 80);
        std::vector<int> all(n);
        for (int i = 0; i < n; ++i) all[i] = i;
        std::vector<GateRec> q;
        for (int i = 0; i < G; ++i) {
            std::shuffle(all.begin(), all.end(), rng);
            const int width = 1 + (int)(rng() % 4);
            std::vector<int> pool(all.begin(), all.begin() + width);
            q.push_back(random_gate(pool, (int)(rng() % 3)));
        }
        // both dense tie rules (0: earliest; 1: most shared qubits)
        const int tie = trial % 2;
        std::vector<PlanItem> plan;
        plan_greedy(q, n, kmax, plan, kMaxDiagQubits, true, 0, 0, tie);
        std::vector<PlanItem> streamed;
        plan_greedy_each(
            q, n, kmax,
            [&](PlanItem &it) {
                streamed.push_back(it);
                return 0;
            },
            kMaxDiagQubits, true, 0, 0, tie);
        // executed order: items in order, members in order
        std::vector<int> order, seen(G, 0);
        for (size_t i = 0; i < plan.size(); ++i) {
            const PlanItem &it = plan[i];
            if (streamed.size() != plan.size() || streamed[i].members != it.members || streamed[i].k != it.k) ++bad;
            uint64_t S = 0;
            for (int j = 0; j < it.k; ++j) S |= 1ull << it.qubits[j];
            for (int gi : it.members) {
                order.push_back(gi);
                seen[gi]++;
                const uint64_t m = q[gi].tmask | q[gi].cmask;
                if (it.fused && !it.diag_block && (m & ~S)) ++bad;
                if (it.diag_block && (!q[gi].diag || (m & ~it.dmask))) ++bad;
            }
            if (it.fused && !it.diag_block) {
                if (it.k > kmax || it.k != __builtin_popcountll(S)) ++bad;
                std::vector<int> Sv(it.qubits, it.qubits + it.k);
                const int D = 1 << it.k;
                std::vector<cd> ref((size_t)D * D, cd(0.0, 0.0));
                for (int d = 0; d < D; ++d) ref[(size_t)d * D + d] = 1.0;
                for (int gi : it.members) ref = matmul(embed(q[gi], Sv), ref, D);
                for (size_t e = 0; e < ref.size(); ++e)
                    if (std::abs(it.m[e] - ref[e]) > 1e-12) {
                        ++bad;
                        break;
                    }
            }
            if (it.diag_block) {
                std::vector<int> Sv;
                for (int b = 0; b < 64; ++b)
                    if ((it.dmask >> b) & 1ull) Sv.push_back(b);
                const int D = 1 << (int)Sv.size();
                std::vector<cd> ref((size_t)D * D, cd(0.0, 0.0));
                for (int d = 0; d < D; ++d) ref[(size_t)d * D + d] = 1.0;
                for (int gi : it.members) ref = matmul(embed(q[gi], Sv), ref, D);
                for (int d = 0; d < D; ++d)
                    if (std::abs(it.dtab[d] - ref[(size_t)d * D + d]) > 1e-12) {
                        ++bad;
                        break;
                    }
            }
        }
        for (int gi = 0; gi < G; ++gi)
            if (seen[gi] != 1) ++bad;
        // program order on every shared qubit
        std::vector<int> at(G);
        for (size_t i = 0; i < order.size(); ++i) at[order[i]] = (int)i;
        for (int a = 0; a < G; ++a)
            for (int b = a + 1; b < G; ++b)
                if (((q[a].tmask | q[a].cmask) & (q[b].tmask | q[b].cmask)) && at[a] > at[b]) {
                    // commuting diagonal gates may be reordered inside one diagonal block
                    bool both_diag_same_block = false;
                    for (const PlanItem &it : plan)
                        if (it.diag_block && std::count(it.members.begin(), it.members.end(), a) &&
                            std::count(it.members.begin(), it.members.end(), b))
                            both_diag_same_block = true;
                    if (!both_diag_same_block) ++bad;
                }
    }
    printf("plan_greedy: %d violations over 60 random circuits\n", bad);
    return bad == 0 ? 0 : 1;
}

int check_perm_plans() {
    int bad = 0, blocks = 0;
    for (int trial = 0; trial < 60; ++trial) {
        // n <= 10 keeps the embedded-matrix check below (2^n x 2^n) quick
        const int n = 6 + trial % 5, kmax = 2 + trial % 4, G = 60 + (int)(rng() % 80);
        const int perm_min = trial % 2 ? 1 : kmax + 1;
        std::vector<int> all(n);
        for (int i = 0; i < n; ++i) all[i] = i;
        std::vector<GateRec> q;
        for (int i = 0; i < G; ++i) {
            std::shuffle(all.begin(), all.end(), rng);
            const int width = 2 + (int)(rng() % 2);
            std::vector<int> pool(all.begin(), all.begin() + width);
            const int r = (int)(rng() % 10);
            q.push_back(r < 6 ? random_gate(pool, 1) : r < 8 ? swap_gate(pool) : random_gate(pool, r == 8 ? 0 : 2));
        }
        std::vector<PlanItem> plan;
        plan_greedy(q, n, kmax, plan, kMaxDiagQubits, true, perm_min);
        std::vector<int> order, seen(G, 0);
        for (const PlanItem &it : plan) {
            for (int gi : it.members) {
                order.push_back(gi);
                seen[gi]++;
            }
            if (!it.perm_block) continue;
            ++blocks;
            std::vector<int> Sv;
            for (int b = 0; b < 64; ++b)
                if ((it.pmask >> b) & 1ull) Sv.push_back(b);
            if ((int)Sv.size() > kMaxPermQubits || (int)Sv.size() < perm_min) ++bad;
            for (int gi : it.members)
                if (!q[gi].perm || ((q[gi].tmask | q[gi].cmask) & ~it.pmask)) ++bad;
            // follow every basis state through the embedded member matrices:
            // each column must hold a single 1, and the last row reached is
            // the table's image
            const int D = 1 << (int)Sv.size();
            std::vector<int> x(D);
            for (int v = 0; v < D; ++v) x[v] = v;
            for (int gi : it.members) {
                const std::vector<cd> E = embed(q[gi], Sv);
                for (int v = 0; v < D; ++v) {
                    int row = -1, ones = 0;
                    for (int r = 0; r < D; ++r) {
                        const cd z = E[(size_t)r * D + x[v]];
                        if (z == cd(1.0, 0.0)) {
                            row = r;
                            ++ones;
                        } else if (z != cd(0.0, 0.0)) {
                            ones = 2;
                        }
                    }
                    if (ones != 1) {
                        ++bad;
                        break;
                    }
                    x[v] = row;
                }
            }
            for (int v = 0; v < D; ++v)
                if ((uint64_t)x[v] != it.ptab[v]) {
                    ++bad;
                    break;
                }
        }
        for (int gi = 0; gi < G; ++gi)
            if (seen[gi] != 1) ++bad;
        std::vector<int> at(G);
        for (size_t i = 0; i < order.size(); ++i) at[order[i]] = (int)i;
        for (int a = 0; a < G; ++a)
            for (int b = a + 1; b < G; ++b)
                if (((q[a].tmask | q[a].cmask) & (q[b].tmask | q[b].cmask)) && at[a] > at[b]) {
                    bool both_diag_same_block = false;
                    for (const PlanItem &it : plan)
                        if (it.diag_block && std::count(it.members.begin(), it.members.end(), a) &&
                            std::count(it.members.begin(), it.members.end(), b))
                            both_diag_same_block = true;
                    if (!both_diag_same_block) ++bad;
                }
    }
    printf("permutation blocks: %d blocks, %d violations over 60 random circuits\n", blocks, bad);
    return bad == 0 && blocks > 0 ? 0 : 1;
}

GateRec h_gate(int b) {
    GateRec g;
    g.t = 1;
    g.targets[0] = b;
    g.tmask = 1ull << b;
    const double h = std::sqrt(0.5);
    g.m = {h, h, h, -h};
    g.kind = GK_DENSE;
    g.perm = perm_map(g, g.pmap);
    return g;
}

GateRec x_gate(int b) {
    GateRec g;
    g.t = 1;
    g.targets[0] = b;
    g.tmask = 1ull << b;
    g.m = {0.0, 1.0, 1.0, 0.0};
    g.kind = GK_X;
    g.perm = perm_map(g, g.pmap);
    return g;
}

int check_product_plans() {
    int bad = 0, items = 0;
    for (int trial = 0; trial < 60; ++trial) {
        const int n = 10 + trial % 7, kmax = 2 + trial % 5, prod_min = kmax + 1;
        std::vector<int> all(n);
        for (int i = 0; i < n; ++i) all[i] = i;
        std::vector<GateRec> q;
        for (int layer = 0; layer < 8; ++layer) {
            const int r = (int)(rng() % 4);
            if (r == 0) {
                // a gate on every qubit: one target, all others as controls
                std::shuffle(all.begin(), all.end(), rng);
                GateRec g = random_gate(std::vector<int>(all.begin(), all.begin() + 1), (int)(rng() % 3));
                for (int j = 1; j < n; ++j) {
                    g.controls.push_back(all[j]);
                    g.cmask |= 1ull << all[j];
                }
                q.push_back(g);
            } else if (r == 3) {
                // a two-qubit gate a dense block can take
                std::shuffle(all.begin(), all.end(), rng);
                q.push_back(random_gate(std::vector<int>(all.begin(), all.begin() + 2), 0));
            } else {
                // one-qubit gates on a random subset of the wires: an H with
                // X before and after at random, and in one layer of six a
                // general gate on one wire
                const bool general = rng() % 6 == 0;
                for (int b = 0; b < n; ++b) {
                    if (rng() % 4 == 0) continue;
                    if (rng() % 2) q.push_back(x_gate(b));
                    q.push_back(general && b == 0 ? random_gate(std::vector<int>{b}, 0) : h_gate(b));
                    if (rng() % 2) q.push_back(x_gate(b));
                }
            }
        }
        const int G = (int)q.size();
        std::vector<PlanItem> plan;
        plan_greedy(q, n, kmax, plan, kMaxDiagQubits, true, 0, prod_min);
        std::vector<int> order, seen(G, 0);
        for (const PlanItem &it : plan)
            for (int gi : it.members) {
                order.push_back(gi);
                seen[gi]++;
            }
        for (int gi = 0; gi < G; ++gi)
            if (seen[gi] != 1) ++bad;
        std::vector<int> at(G);
        for (size_t i = 0; i < order.size(); ++i) at[order[i]] = (int)i;
        for (int a = 0; a < G; ++a)
            for (int b = a + 1; b < G; ++b)
                if (((q[a].tmask | q[a].cmask) & (q[b].tmask | q[b].cmask)) && at[a] > at[b]) {
                    bool both_diag_same_block = false;
                    for (const PlanItem &it : plan)
                        if (it.diag_block && std::count(it.members.begin(), it.members.end(), a) &&
                            std::count(it.members.begin(), it.members.end(), b))
                            both_diag_same_block = true;
                    if (!both_diag_same_block) ++bad;
                }
        for (const PlanItem &it : plan) {
            if (!it.prod_block) continue;
            ++items;
            if (__builtin_popcountll(it.qmask_prod) < prod_min) ++bad;
            std::vector<int> wires;
            for (int b = 0; b < n; ++b)
                if ((it.qmask_prod >> b) & 1ull) wires.push_back(b);
            if (it.pm.size() != 4 * wires.size()) {
                ++bad;
                continue;
            }
            // members on a wire outside the item: their product is the identity
            for (int b = 0; b < n; ++b) {
                if ((it.qmask_prod >> b) & 1ull) continue;
                std::vector<cd> ref = {1.0, 0.0, 0.0, 1.0};
                for (int gi : it.members)
                    if (q[gi].targets[0] == b) ref = matmul(q[gi].m, ref, 2);
                if (std::abs(ref[0] - 1.0) > 1e-12 || std::abs(ref[1]) > 1e-12 || std::abs(ref[2]) > 1e-12 ||
                    std::abs(ref[3] - 1.0) > 1e-12)
                    ++bad;
            }
            for (int gi : it.members)
                if (q[gi].t != 1 || !q[gi].controls.empty()) ++bad;
            for (size_t w = 0; w < wires.size(); ++w) {
                const int b = wires[w];
                std::vector<cd> ref = {1.0, 0.0, 0.0, 1.0};
                int last = -1;
                for (int gi : it.members) {
                    const GateRec &g = q[gi];
                    if (g.targets[0] != b) continue;
                    ref = matmul(g.m, ref, 2);
                    last = std::max(last, gi);
                }
                for (int e = 0; e < 4; ++e)
                    if (std::abs(it.pm[4 * w + e] - ref[e]) > 1e-12) ++bad;
                // c times a +-1 matrix with orthogonal rows
                const cd *M = &it.pm[4 * w];
                const double c = std::abs(M[0]);
                for (int e = 0; e < 4; ++e)
                    if (std::abs(M[e].imag()) > 1e-12 || std::abs(std::abs(M[e].real()) - c) > 1e-12) ++bad;
                if (std::abs(M[0].real() * M[2].real() + M[1].real() * M[3].real()) > 1e-12) ++bad;
                // the wire's next gate after the item is wider than kmax, or none
                for (int gi = last + 1; gi < G; ++gi)
                    if (((q[gi].tmask | q[gi].cmask) >> b) & 1ull) {
                        if (__builtin_popcountll(q[gi].tmask | q[gi].cmask) <= kmax) ++bad;
                        break;
                    }
            }
        }
    }
    printf("product items: %d items, %d violations over 60 random circuits\n", items, bad);
    // Grover's search (3 iterations on 20 qubits): the first H layer and
    // every layer between two many-controlled Z are product items; a U3 +
    // CNOT brickwork (every wire continues into a CNOT) forms none
    {
        const int n = 20;
        const uint64_t marked = 0x5a5a5ull;
        std::vector<GateRec> q;
        auto mcz = [&]() {
            GateRec g;
            g.t = 1;
            g.targets[0] = n - 1;
            g.tmask = 1ull << (n - 1);
            g.m = {1.0, 0.0, 0.0, -1.0};
            g.kind = GK_DIAG1;
            g.diag = true;
            for (int c = 0; c < n - 1; ++c) {
                g.controls.push_back(c);
                g.cmask |= 1ull << c;
            }
            g.perm = perm_map(g, g.pmap);
            return g;
        };
        for (int b = 0; b < n; ++b) q.push_back(h_gate(b));
        for (int it = 0; it < 3; ++it) {
            for (int b = 0; b < n; ++b)
                if (!((marked >> b) & 1)) q.push_back(x_gate(b));
            q.push_back(mcz());
            for (int b = 0; b < n; ++b)
                if (!((marked >> b) & 1)) q.push_back(x_gate(b));
            for (int b = 0; b < n; ++b) q.push_back(h_gate(b));
            for (int b = 0; b < n; ++b) q.push_back(x_gate(b));
            q.push_back(mcz());
            for (int b = 0; b < n; ++b) q.push_back(x_gate(b));
            for (int b = 0; b < n; ++b) q.push_back(h_gate(b));
        }
        std::vector<PlanItem> plan;
        plan_greedy(q, n, 6, plan, kMaxDiagQubits, true, perm_min_width(QSIM_C64, 6), 7);
        int prod = 0, plain = 0;
        for (const PlanItem &it : plan) {
            if (it.prod_block && __builtin_popcountll(it.qmask_prod) == n) ++prod;
            if (!it.fused) ++plain;
        }
        const bool grover_ok = prod == 7 && plain == 6 && plan.size() == 13;
        std::vector<GateRec> bw;
        for (int l = 0; l < 10; ++l) {
            for (int b = 0; b < n; ++b) {
                GateRec g = random_gate(std::vector<int>{b}, 0);
                g.controls.clear();
                g.cmask = 0;
                bw.push_back(g);
            }
            for (int b = l % 2; b + 1 < n; b += 2) {
                GateRec g = x_gate(b + 1);
                g.controls.push_back(b);
                g.cmask = 1ull << b;
                g.perm = perm_map(g, g.pmap);
                bw.push_back(g);
            }
        }
        std::vector<PlanItem> pbw, pbw0;
        plan_greedy(bw, n, 6, pbw, kMaxDiagQubits, true, perm_min_width(QSIM_C64, 6), 7);
        plan_greedy(bw, n, 6, pbw0, kMaxDiagQubits, true, perm_min_width(QSIM_C64, 6), 0);
        int bw_prod = 0;
        for (const PlanItem &it : pbw) bw_prod += it.prod_block;
        const bool bw_ok = bw_prod == 0 && pbw.size() == pbw0.size();
        printf("Grover 20 qubits, 3 iterations: %d items (%d full-width product, %d plain); brickwork: %zu items, "
               "%d product (%zu without product passes)\n",
               (int)plan.size(), prod, plain, pbw.size(), bw_prod, pbw0.size());
        if (!grover_ok || !bw_ok) ++bad;
    }
    return bad == 0 && items > 0 ? 0 : 1;
}

int check_qft_plan() {
    const int n = 30;
    std::vector<GateRec> q;
    for (int j = n - 1; j >= 0; --j) {
        q.push_back(h_gate(j));
        for (int k = j - 1; k >= 0; --k) {
            GateRec g;
            g.t = 1;
            g.targets[0] = j;
            g.tmask = 1ull << j;
            g.controls.push_back(k);
            g.cmask = 1ull << k;
            g.m = {1.0, 0.0, 0.0, std::polar(1.0, M_PI / (double)(1ull << (j - k)))};
            g.kind = GK_PHASE;
            g.diag = true;
            g.perm = perm_map(g, g.pmap);
            q.push_back(g);
        }
    }
    for (int i = 0; i < n / 2; ++i) q.push_back(swap_gate(std::vector<int>{i, n - 1 - i}));
    std::vector<PlanItem> plan;
    plan_greedy(q, n, 6, plan, kMaxDiagQubits, true, perm_min_width(QSIM_C64, 6), 7);
    int full = 0, seen = 0;
    for (const PlanItem &it : plan) {
        if (it.diag_block && it.members.size() == 36) ++full;
        seen += (int)it.members.size();
    }
    printf("QFT 30 qubits: %zu items, %d diagonal blocks of 36 phase gates\n", plan.size(), full);
    const bool qft_ok = plan.size() == 20 && full == 10 && seen == (int)q.size();
    // the circuit of the paper's Fig. 7: H on all, a controlled-Rz chain, H
    // on all; tie rule 0 leaves the chain gates across block edges behind
    std::vector<GateRec> f;
    for (int b = 0; b < n; ++b) f.push_back(h_gate(b));
    for (int i = 0; i + 1 < n; ++i) {
        GateRec g;
        g.t = 1;
        g.targets[0] = i + 1;
        g.tmask = 1ull << (i + 1);
        g.controls.push_back(i);
        g.cmask = 1ull << i;
        const double phi = 0.1 * (i + 1);
        g.m = {std::polar(1.0, -phi / 2), 0.0, 0.0, std::polar(1.0, phi / 2)};
        g.kind = GK_DIAG1;
        g.diag = true;
        g.perm = perm_map(g, g.pmap);
        f.push_back(g);
    }
    for (int b = 0; b < n; ++b) f.push_back(h_gate(b));
    std::vector<PlanItem> f0, f1;
    plan_greedy(f, n, 6, f0, kMaxDiagQubits, true, perm_min_width(QSIM_C64, 6), 7, 0);
    plan_greedy(f, n, 6, f1, kMaxDiagQubits, true, perm_min_width(QSIM_C64, 6), 7, 1);
    printf("Fig. 7 circuit, 30 qubits: %zu items with tie rule 0, %zu with tie rule 1\n", f0.size(), f1.size());
    return qft_ok && f1.size() == 6 && f0.size() > f1.size() ? 0 : 1;
}

}  // namespace

int main() {
    const int a = check_block_matrix();
    const int b = check_plans();
    const int c = check_perm_plans();
    const int d = check_product_plans();
    const int e = check_qft_plan();
    return a | b | c | d | e;
}
