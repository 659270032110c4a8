// The paper's hybrid pipeline, host side (Sec. 3.3 "Map on CPU" and the
// matrix preparation of "Reduce on GPU", measured in Sec. 4.1): a baseline
// for the GPU path, not the oracle and not on the product path.
//   map:    each document is counted into its own dictionary, documents
//           spread over threads (the paper's @floop over documents);
//   group:  one dictionary word -> the counts of the word in every document
//           that has it (no addition yet), built by one thread per hash range;
//   matrix: a zero-filled row-major uint32 matrix with one row per word and
//           as many columns as the longest count list, each row holding its
//           word's counts from column 0.
// The matrix then goes to the GPU, whose row sums are the reduce
// (wc_row_sums in the CUDA library).  Words follow the same letters-only rule
// as everything else here.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

inline bool letter(uint8_t b) { return (uint8_t)((b | 0x20) - 'a') < 26 && b < 0x80; }

using DocMap = std::unordered_map<std::string, uint32_t>;

struct Hybrid {
    std::vector<std::string> words;            // row r's word
    std::vector<std::vector<uint32_t>> lists;  // row r's counts, one per document that has the word
    uint64_t cols = 0, word_bytes = 0;
};

void count_doc(const uint8_t *t, uint64_t lo, uint64_t hi, DocMap &m) {
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

extern "C" {

// Map + group; returns a handle (null on bad arguments) and the matrix shape.
void *hybrid_map(const uint8_t *text, const uint64_t *offs, uint32_t ndocs, int threads, uint64_t *rows,
                 uint64_t *cols, uint64_t *word_bytes) {
    if (threads < 1) threads = 1;
    if (ndocs && (!text || !offs)) return nullptr;
    std::vector<DocMap> docs(ndocs);
    {
        std::vector<std::thread> th;
        for (int p = 0; p < threads; p++)
            th.emplace_back([&, p] {
                for (uint32_t d = (uint32_t)p; d < ndocs; d += (uint32_t)threads) count_doc(text, offs[d], offs[d + 1], docs[d]);
            });
        for (auto &x : th) x.join();
    }
    // group: thread r owns the words whose hash falls in range r
    std::vector<std::unordered_map<std::string, std::vector<uint32_t>>> part((size_t)threads);
    {
        std::vector<std::thread> th;
        for (int r = 0; r < threads; r++)
            th.emplace_back([&, r] {
                std::hash<std::string> h;
                for (auto &m : docs)
                    for (auto &kv : m)
                        if ((int)(h(kv.first) % (size_t)threads) == r) part[r][kv.first].push_back(kv.second);
            });
        for (auto &x : th) x.join();
    }
    Hybrid *hy = new Hybrid();
    for (auto &p : part)
        for (auto &kv : p) {
            hy->cols = std::max<uint64_t>(hy->cols, kv.second.size());
            hy->word_bytes += kv.first.size();
            hy->words.push_back(kv.first);
            hy->lists.push_back(std::move(kv.second));
        }
    if (rows) *rows = hy->words.size();
    if (cols) *cols = hy->cols;
    if (word_bytes) *word_bytes = hy->word_bytes;
    return hy;
}

// Fills the padded matrix (rows x cols uint32, row-major; zeroed here) with
// `threads` threads, and optionally the words (back to back) and their
// offsets (rows + 1).
int hybrid_fill(void *handle, uint32_t *matrix, int threads, uint8_t *words, uint64_t *word_offs) {
    Hybrid *hy = static_cast<Hybrid *>(handle);
    if (!hy) return -1;
    const uint64_t rows = hy->words.size(), cols = hy->cols;
    if (threads < 1) threads = 1;
    if (matrix) {
        std::vector<std::thread> th;
        for (int p = 0; p < threads; p++)
            th.emplace_back([&, p] {
                const uint64_t r0 = rows * (uint64_t)p / (uint64_t)threads, r1 = rows * (uint64_t)(p + 1) / (uint64_t)threads;
                for (uint64_t r = r0; r < r1; r++) {
                    uint32_t *row = matrix + r * cols;
                    const std::vector<uint32_t> &l = hy->lists[r];
                    std::memcpy(row, l.data(), l.size() * 4);
                    std::memset(row + l.size(), 0, (cols - l.size()) * 4);
                }
            });
        for (auto &x : th) x.join();
    }
    if (words || word_offs) {
        uint64_t o = 0;
        for (uint64_t r = 0; r < rows; r++) {
            if (word_offs) word_offs[r] = o;
            if (words) std::memcpy(words + o, hy->words[r].data(), hy->words[r].size());
            o += hy->words[r].size();
        }
        if (word_offs) word_offs[rows] = o;
    }
    return 0;
}

void hybrid_free(void *handle) { delete static_cast<Hybrid *>(handle); }

}  // extern "C"
