// Paper-style parallel CPU word count, a baseline for the GPU path (not the
// oracle, and not on the product path).  It follows the paper's multicore
// map (Sec. 3.1: each thread builds its own dictionary over its share of the
// input, Julia's @floop over documents) and reduce (Sec. 3.3: the
// dictionaries are summed), here over one large text: the text is cut into
// one piece per thread after a non-letter byte, each thread counts its piece
// into its own hash map, the maps are merged by one thread per hash range,
// and the merged table is sorted by (count desc, word asc).  Words follow
// the same letters-only rule as everything else here: maximal runs of ASCII
// letters, lowercased.
#include <algorithm>
#include <cstdint>
#include <string>
#include <string_view>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

inline bool letter(uint8_t b) { return (uint8_t)((b | 0x20) - 'a') < 26 && b < 0x80; }

using Map = std::unordered_map<std::string, uint64_t>;

void count_piece(const uint8_t *t, uint64_t lo, uint64_t hi, Map &m) {
    std::string w;
    uint64_t i = lo;
    while (i < hi) {
        while (i < hi && !letter(t[i])) i++;
        if (i >= hi) break;
        w.clear();
        while (i < hi && letter(t[i])) w.push_back((char)(t[i++] | 0x20));
        ++m[w];
    }
}

}  // namespace

extern "C" int cpu_parallel_count(const uint8_t *text, uint64_t n, int threads, uint64_t *out_distinct,
                                  uint64_t *out_tokens, uint64_t *out_top_count) {
    if (threads < 1) threads = 1;
    // pieces cut after a non-letter byte: no word spans two pieces
    std::vector<uint64_t> cut{0};
    for (int p = 1; p < threads; p++) {
        uint64_t c = std::max<uint64_t>(cut.back(), n * (uint64_t)p / (uint64_t)threads);
        while (c < n && c > 0 && letter(text[c - 1]) && letter(text[c])) c++;
        cut.push_back(c);
    }
    cut.push_back(n);
    const int np = (int)cut.size() - 1;
    std::vector<Map> maps((size_t)np);
    {
        std::vector<std::thread> th;
        for (int p = 0; p < np; p++) th.emplace_back(count_piece, text, cut[p], cut[p + 1], std::ref(maps[p]));
        for (auto &x : th) x.join();
    }
    // merge: thread r owns the words whose hash falls in range r
    std::vector<Map> merged((size_t)threads);
    {
        std::vector<std::thread> th;
        for (int r = 0; r < threads; r++)
            th.emplace_back([&, r] {
                std::hash<std::string> h;
                for (auto &m : maps)
                    for (auto &kv : m)
                        if ((int)(h(kv.first) % (size_t)threads) == r) merged[r][kv.first] += kv.second;
            });
        for (auto &x : th) x.join();
    }
    std::vector<std::pair<uint64_t, const std::string *>> all;
    uint64_t tokens = 0;
    for (auto &m : merged)
        for (auto &kv : m) {
            all.emplace_back(kv.second, &kv.first);
            tokens += kv.second;
        }
    std::sort(all.begin(), all.end(), [](const auto &a, const auto &b) {
        return a.first != b.first ? a.first > b.first : *a.second < *b.second;
    });
    if (out_distinct) *out_distinct = all.size();
    if (out_tokens) *out_tokens = tokens;
    if (out_top_count) *out_top_count = all.empty() ? 0 : all[0].first;
    return 0;
}
