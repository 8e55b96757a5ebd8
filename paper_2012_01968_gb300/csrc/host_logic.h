// Host-side scheduling logic of the library, free of CUDA so that it can be
// compiled and tested on its own: how the host-buffer call splits its data,
// how a batch submission groups and places its jobs, and the first-fit
// allocator of the serving arena.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

namespace ntt {
namespace host {

// A piece of a [batch][L][N] array: limbs [first, first + count), whose limb
// i uses prime prime0 + (i % lview).
struct Segment {
    uint32_t first, count, prime0, lview;
};

// Split batch x L limbs into at most max_segments pieces: limb ranges inside
// each polynomial when there are fewer polynomials than pieces (so that one
// polynomial still gives several pieces), else groups of whole polynomials.
inline std::vector<Segment> split_segments(uint32_t batch, uint32_t L, uint32_t max_segments)
{
    std::vector<Segment> segs;
    if (batch == 0 || L == 0 || max_segments == 0) return segs;
    if (batch >= max_segments) {
        const uint32_t per = (batch + max_segments - 1) / max_segments;
        for (uint32_t b0 = 0; b0 < batch; b0 += per) {
            const uint32_t nb = batch - b0 < per ? batch - b0 : per;
            segs.push_back(Segment{b0 * L, nb * L, 0, L});
        }
    } else {
        const uint32_t pieces = max_segments / batch;         // batch * pieces <= max_segments
        const uint32_t c = (L + pieces - 1) / pieces;
        for (uint32_t b0 = 0; b0 < batch; ++b0)
            for (uint32_t r = 0; r < L; r += c) {
                const uint32_t cnt = L - r < c ? L - r : c;
                segs.push_back(Segment{b0 * L + r, cnt, r, cnt});
            }
    }
    return segs;
}

// Does any pair of half-open byte ranges overlap?
inline bool any_overlap(std::vector<std::pair<uintptr_t, uintptr_t>> ranges)
{
    std::sort(ranges.begin(), ranges.end());
    for (size_t i = 1; i < ranges.size(); ++i)
        if (ranges[i].first < ranges[i - 1].second) return true;
    return false;
}

// One launch of a batch submission: jobs (indices into the submission) that
// share a key (size, direction, OT stages), at most max_jobs of them.
struct Chunk {
    std::vector<uint32_t> jobs;
    uint64_t limbs = 0;
    double work = 0;              // limbs x N, to balance the streams
    std::tuple<uint32_t, uint32_t, uint32_t> key{};
};

// Group jobs by key (in key order, jobs in submission order within a key),
// cut each group into chunks of at most max_jobs, and order the chunks by
// decreasing work.  keys[i], limbs[i], size[i] (N) describe job i.
inline std::vector<Chunk> make_chunks(const std::vector<std::tuple<uint32_t, uint32_t, uint32_t>>& keys,
                                      const std::vector<uint64_t>& limbs, const std::vector<uint64_t>& size,
                                      uint32_t max_jobs)
{
    std::map<std::tuple<uint32_t, uint32_t, uint32_t>, std::vector<uint32_t>> groups;
    for (uint32_t i = 0; i < (uint32_t)keys.size(); ++i) groups[keys[i]].push_back(i);
    std::vector<Chunk> chunks;
    for (auto& g : groups) {
        const auto& idx = g.second;
        for (size_t k = 0; k < idx.size(); k += max_jobs) {
            Chunk c;
            c.key = g.first;
            for (size_t m = k; m < idx.size() && m < k + max_jobs; ++m) {
                c.jobs.push_back(idx[m]);
                c.limbs += limbs[idx[m]];
                c.work += (double)limbs[idx[m]] * (double)size[idx[m]];
            }
            chunks.push_back(std::move(c));
        }
    }
    std::stable_sort(chunks.begin(), chunks.end(), [](const Chunk& x, const Chunk& y) { return x.work > y.work; });
    return chunks;
}

// Longest-first placement: each work item (in the given order) goes to the
// least loaded of `streams` streams; returns the stream of each item.
inline std::vector<int> place_least_loaded(const std::vector<double>& work, int streams)
{
    std::vector<double> load(streams > 0 ? streams : 1, 0.0);
    std::vector<int> at;
    at.reserve(work.size());
    for (double w : work) {
        int best = 0;
        for (int k = 1; k < (int)load.size(); ++k)
            if (load[k] < load[best]) best = k;
        load[best] += w;
        at.push_back(best);
    }
    return at;
}

// First-fit allocator over [0, size) in 256-byte granules; freed ranges are
// merged with free neighbours.
class Arena {
public:
    void reset(size_t size)
    {
        free_.clear();
        size = size & ~(size_t)255;
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    const std::map<size_t, size_t>& free_ranges() const { return free_; }

private:
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
    std::map<size_t, size_t> free_;
};

// Configurations the autotuner times for N = 2^n, as plan option codes
// (kernel 1 FUSED, 2 PER_PASS, 3 RADIX2, 4 HIGH_RADIX (radix 16); twiddle 1
// TABLE, 2 OT with ot_stages 1 or 2; geometry 0 .. geometries-1).  Two-pass
// sizes (n >= 13): every geometry x {FUSED, PER_PASS} x {TABLE, OT1, OT2},
// then RADIX2 and HIGH_RADIX with table twiddles.  One-pass sizes: the
// one-pass kernel (kernel 0 = AUTO), RADIX2 and HIGH_RADIX, and for
// n = 10 .. 12 the cluster kernel (kernel 5 CLUSTER).
struct TuneCandidate {
    uint32_t kernel, twiddle_mode, ot_stages, geometry;
};
inline std::vector<TuneCandidate> tune_candidates(uint32_t n, uint32_t geometries, uint32_t single_pass_max)
{
    std::vector<TuneCandidate> out;
    if (n <= single_pass_max) {
        out.push_back(TuneCandidate{0, 1, 0, 0});
        out.push_back(TuneCandidate{3, 1, 0, 0});
        out.push_back(TuneCandidate{4, 1, 0, 0});
        if (n >= 10 && n <= 12) out.push_back(TuneCandidate{5, 1, 0, 0});   // the cluster kernel's sizes
        return out;
    }
    for (uint32_t g = 0; g < geometries; ++g)
        for (uint32_t k = 1; k <= 2; ++k) {
            out.push_back(TuneCandidate{k, 1, 0, g});
            out.push_back(TuneCandidate{k, 2, 1, g});
            out.push_back(TuneCandidate{k, 2, 2, g});
        }
    out.push_back(TuneCandidate{3, 1, 0, 0});
    out.push_back(TuneCandidate{4, 1, 0, 0});
    return out;
}

// Index of the fastest timed candidate by forward + inverse time (ties: the
// earlier one), or -1 when none was timed (ok[i] false for all).
inline int tune_pick(const std::vector<double>& fwd_us, const std::vector<double>& inv_us,
                     const std::vector<bool>& ok)
{
    int best = -1;
    for (size_t i = 0; i < fwd_us.size(); ++i) {
        if (!ok[i]) continue;
        if (best < 0 || fwd_us[i] + inv_us[i] < fwd_us[(size_t)best] + inv_us[(size_t)best]) best = (int)i;
    }
    return best;
}

}  // namespace host
}  // namespace ntt
