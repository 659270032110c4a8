// Word-frequency oracle: a plain, single-threaded CPU implementation of what
// the counting path computes.  TEST INFRASTRUCTURE ONLY: it is used by the
// tests, by the smoke check and by the benchmark's CPU-baseline arm, never by
// the product path.  It shares no code with the CUDA library.
//
// What it computes (the plain definition, written out):
//   Normalisation and map (Sec. 2 and Sec. 3.1 of the paper: punctuation is
//   removed and text lowercased so "Dog" and "dog." are the same word, then
//   each document is split into words).  Here the rule is fixed as: a word is
//   a maximal run of ASCII letters [A-Za-z]; each letter is lowercased; every
//   other byte (digits, punctuation, whitespace, bytes >= 0x80) separates
//   words; a document edge separates words.
//   Reduce (Sec. 3.1 per-document dictionaries, Sec. 3.2/3.3 summing the
//   per-document counts of each key): count_d(w) = number of words of
//   document d equal to w; count_class(c, w) = sum of count_d(w) over the
//   documents of class c; count_global(w) = sum over all documents.
//   Output order: count descending, then word bytes ascending (memcmp order,
//   a proper prefix first).
//   Class ratio ranking (the distinguishing-word study of Sec. 4.3, made
//   exact): within class c, words with cin >= 1 are ranked by cin/cout
//   descending where cout = count_global - cin (cout = 0 ranks above every
//   finite ratio), then cin descending, then word ascending.  Ratios are
//   compared by cross-multiplication in 128-bit integers.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

typedef std::vector<std::pair<std::string, uint64_t>> Table;

static bool is_letter(uint8_t b) { return (b >= 'A' && b <= 'Z') || (b >= 'a' && b <= 'z'); }
static char lower(uint8_t b) { return (b >= 'A' && b <= 'Z') ? (char)(b - 'A' + 'a') : (char)b; }

// Splits bytes [p, p+n) into words and adds one per occurrence to m.
static void count_words(const uint8_t* p, uint64_t n, std::unordered_map<std::string, uint64_t>& m) {
    uint64_t i = 0;
    while (i < n) {
        if (!is_letter(p[i])) { i++; continue; }
        std::string w;
        while (i < n && is_letter(p[i])) { w.push_back(lower(p[i])); i++; }
        m[w] += 1;
    }
}

static bool by_count_then_word(const std::pair<std::string, uint64_t>& a, const std::pair<std::string, uint64_t>& b) {
    if (a.second != b.second) return a.second > b.second;
    return a.first < b.first;  // std::string compares bytes as unsigned char, prefix first
}

static Table sorted_table(const std::unordered_map<std::string, uint64_t>& m) {
    Table t(m.begin(), m.end());
    std::sort(t.begin(), t.end(), by_count_then_word);
    return t;
}

struct Result {
    std::vector<Table> docs;
    std::vector<Table> classes;
    Table global;
    std::vector<std::unordered_map<std::string, uint64_t>> class_maps;
    std::unordered_map<std::string, uint64_t> global_map;
};

}  // namespace

extern "C" {

// Counts every document; per-document tables are kept only if keep_docs != 0.
// classes may be NULL (then nclasses must be 0).
void* oracle_count(const uint8_t* text, const uint64_t* offsets, uint32_t ndocs,
                   const uint32_t* classes, uint32_t nclasses, int keep_docs) {
    Result* r = new Result();
    r->class_maps.resize(nclasses);
    if (keep_docs) r->docs.resize(ndocs);
    for (uint32_t d = 0; d < ndocs; d++) {
        std::unordered_map<std::string, uint64_t> m;
        count_words(text + offsets[d], offsets[d + 1] - offsets[d], m);
        for (const auto& kv : m) {
            r->global_map[kv.first] += kv.second;
            if (classes) r->class_maps[classes[d]][kv.first] += kv.second;
        }
        if (keep_docs) r->docs[d] = sorted_table(m);
    }
    r->global = sorted_table(r->global_map);
    for (uint32_t c = 0; c < nclasses; c++) r->classes.push_back(sorted_table(r->class_maps[c]));
    return r;
}

// Sums already-counted tables word by word (the reduce of Sec. 3.3: "the",
// counted 10, 4 and 3 times in three documents, reduces to 17).
// Tables are given as concatenated word bytes + offsets + counts.
void* oracle_merge(uint32_t ntables, const uint8_t* const* words, const uint64_t* const* offs,
                   const uint64_t* const* counts, const uint64_t* sizes) {
    Result* r = new Result();
    for (uint32_t t = 0; t < ntables; t++)
        for (uint64_t i = 0; i < sizes[t]; i++) {
            std::string w((const char*)words[t] + offs[t][i], offs[t][i + 1] - offs[t][i]);
            r->global_map[w] += counts[t][i];
        }
    r->global = sorted_table(r->global_map);
    return r;
}

static const Table* pick(void* h, int kind, uint32_t idx) {
    Result* r = (Result*)h;
    if (kind == 0) return idx < r->docs.size() ? &r->docs[idx] : nullptr;
    if (kind == 1) return idx < r->classes.size() ? &r->classes[idx] : nullptr;
    return &r->global;
}

// kind: 0 = document, 1 = class, 2 = global.  Returns -1 for a bad index.
int64_t oracle_table_size(void* h, int kind, uint32_t idx, uint64_t* word_bytes, uint64_t* tokens) {
    const Table* t = pick(h, kind, idx);
    if (!t) return -1;
    uint64_t b = 0, s = 0;
    for (const auto& kv : *t) { b += kv.first.size(); s += kv.second; }
    if (word_bytes) *word_bytes = b;
    if (tokens) *tokens = s;
    return (int64_t)t->size();
}

// Writes the sorted table: words back to back, offs[n+1], counts[n].
int oracle_table_export(void* h, int kind, uint32_t idx, uint8_t* words, uint64_t* offs, uint64_t* counts) {
    const Table* t = pick(h, kind, idx);
    if (!t) return -1;
    uint64_t p = 0;
    for (size_t i = 0; i < t->size(); i++) {
        const auto& kv = (*t)[i];
        offs[i] = p;
        memcpy(words + p, kv.first.data(), kv.first.size());
        p += kv.first.size();
        counts[i] = kv.second;
    }
    offs[t->size()] = p;
    return 0;
}

// Top-k words of class c by the ratio of in-class to out-of-class count.
// Writes up to k indices into the class table's sorted order (out_idx) and
// the pair (cin, cout) per word; returns how many were written.
int64_t oracle_ratio_topk(void* h, uint32_t c, uint32_t k, uint64_t* out_idx, uint64_t* out_cin, uint64_t* out_cout) {
    Result* r = (Result*)h;
    if (c >= r->classes.size()) return -1;
    const Table& t = r->classes[c];
    struct Item { uint64_t idx, cin, cout; };
    std::vector<Item> items;
    for (size_t i = 0; i < t.size(); i++) {
        uint64_t cin = t[i].second;
        uint64_t g = r->global_map.at(t[i].first);
        items.push_back({(uint64_t)i, cin, g - cin});
    }
    auto better = [&](const Item& a, const Item& b) {
        // a/acout vs b/bcout with cout = 0 meaning +infinity
        bool ainf = a.cout == 0, binf = b.cout == 0;
        if (ainf != binf) return ainf;
        if (!ainf) {
            unsigned __int128 lhs = (unsigned __int128)a.cin * b.cout;
            unsigned __int128 rhs = (unsigned __int128)b.cin * a.cout;
            if (lhs != rhs) return lhs > rhs;
        }
        if (a.cin != b.cin) return a.cin > b.cin;
        return t[a.idx].first < t[b.idx].first;
    };
    std::sort(items.begin(), items.end(), better);
    uint64_t n = std::min<uint64_t>(k, items.size());
    for (uint64_t i = 0; i < n; i++) { out_idx[i] = items[i].idx; out_cin[i] = items[i].cin; out_cout[i] = items[i].cout; }
    return (int64_t)n;
}

void oracle_free(void* h) { delete (Result*)h; }

}  // extern "C"
