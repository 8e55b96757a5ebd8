// Test driver for the library's CUDA-free host logic (csrc/host_logic.h):
// reads commands on stdin, prints results on stdout, one line per command.
#include <cstdio>
#include <iostream>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "host_logic.h"

using namespace ntt::host;

int main()
{
    std::string cmd;
    while (std::cin >> cmd) {
        if (cmd == "segments") {
            uint32_t b, L, m;
            std::cin >> b >> L >> m;
            const auto s = split_segments(b, L, m);
            std::printf("%zu", s.size());
            for (const auto& g : s) std::printf(" %u %u %u %u", g.first, g.count, g.prime0, g.lview);
            std::printf("\n");
        } else if (cmd == "arena") {
            size_t size;
            int nops;
            std::cin >> size >> nops;
            Arena a;
            a.reset(size);
            for (int i = 0; i < nops; ++i) {
                char op;
                std::cin >> op;
                if (op == 'a') {
                    size_t bytes, off = 0;
                    std::cin >> bytes;
                    const bool ok = a.alloc(bytes, &off);
                    std::printf("%d %zu ", ok ? 1 : 0, ok ? off : (size_t)0);
                } else {
                    size_t off, bytes;
                    std::cin >> off >> bytes;
                    a.release(off, bytes);
                    std::printf("r ");
                }
            }
            std::printf("| %zu", a.free_ranges().size());
            for (const auto& kv : a.free_ranges()) std::printf(" %zu %zu", kv.first, kv.second);
            std::printf("\n");
        } else if (cmd == "chunks") {
            int nj;
            uint32_t maxj;
            std::cin >> nj >> maxj;
            std::vector<std::tuple<uint32_t, uint32_t, uint32_t>> keys(nj);
            std::vector<uint64_t> limbs(nj), size(nj);
            for (int i = 0; i < nj; ++i) {
                uint32_t a, b, c;
                std::cin >> a >> b >> c >> limbs[i] >> size[i];
                keys[i] = std::make_tuple(a, b, c);
            }
            const auto ch = make_chunks(keys, limbs, size, maxj);
            std::printf("%zu", ch.size());
            for (const auto& c : ch) {
                std::printf(" ; %u %u %u %llu %.1f %zu", std::get<0>(c.key), std::get<1>(c.key), std::get<2>(c.key),
                            (unsigned long long)c.limbs, c.work, c.jobs.size());
                for (uint32_t j : c.jobs) std::printf(" %u", j);
            }
            std::printf("\n");
        } else if (cmd == "place") {
            int nw, streams;
            std::cin >> nw >> streams;
            std::vector<double> w(nw);
            for (auto& x : w) std::cin >> x;
            for (int k : place_least_loaded(w, streams)) std::printf("%d ", k);
            std::printf("\n");
        } else if (cmd == "overlap") {
            int n;
            std::cin >> n;
            std::vector<std::pair<uintptr_t, uintptr_t>> r(n);
            for (auto& x : r) std::cin >> x.first >> x.second;
            std::printf("%d\n", any_overlap(r) ? 1 : 0);
        } else if (cmd == "tune") {
            uint32_t n, geometries, single_max;
            std::cin >> n >> geometries >> single_max;
            for (const auto& c : tune_candidates(n, geometries, single_max))
                std::printf("%u %u %u %u ; ", c.kernel, c.twiddle_mode, c.ot_stages, c.geometry);
            std::printf("\n");
        } else if (cmd == "pick") {
            int m;
            std::cin >> m;
            std::vector<double> f(m), v(m);
            std::vector<bool> ok(m);
            for (int i = 0; i < m; ++i) {
                int o;
                std::cin >> f[i] >> v[i] >> o;
                ok[i] = o != 0;
            }
            std::printf("%d\n", tune_pick(f, v, ok));
        }
    }
    return 0;
}
