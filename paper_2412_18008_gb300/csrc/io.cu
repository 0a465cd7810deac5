// Saving a built hierarchy to a file and loading it back onto the device
// (ch_save / ch_load), and one-to-many queries (ch_query_one_to_many).
//
// File layout (little-endian): an 8-byte magic, a fixed header of sizes,
// then the arrays in a fixed order: rank, perm, level, priority, both rank-
// ordered CSRs (offsets, adjacency), the shortcut log with its rounds, the
// per-round counters and times, and the build summary. Learned-priority
// traces are not saved.

#include <cstdio>
#include <cstring>
#include <memory>
#include <new>

#include "handle.cuh"

namespace gbch {
namespace {

constexpr char kMagic[8] = {'G', 'B', 'C', 'H', '0', '0', '0', '1'};

struct FileHeader {
    uint32_t n, hop_limit;
    uint64_t m_input, n_up, n_down, n_shortcuts, rounds, core_size;
    uint32_t nstat, ntime;  // per-round widths, checked on load
};

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) std::fclose(f);
    }
};

void put(FILE *f, const void *p, size_t bytes) {
    if (bytes && std::fwrite(p, 1, bytes, f) != bytes) throw Error{CH_EINVAL, "write failed"};
}

void get(FILE *f, void *p, size_t bytes) {
    if (bytes && std::fread(p, 1, bytes, f) != bytes) throw Error{CH_EINVAL, "file is truncated"};
}

template <class T>
void put_dev(FILE *f, const DevBuf<T> &b, uint64_t count) {
    if (!count) return;
    std::vector<T> h(count);
    CH_CUDA_TRY(cudaMemcpy(h.data(), b.ptr, count * sizeof(T), cudaMemcpyDeviceToHost));
    put(f, h.data(), count * sizeof(T));
}

template <class T>
std::vector<T> get_vec(FILE *f, uint64_t count) {
    std::vector<T> h(count);
    get(f, h.data(), count * sizeof(T));
    return h;
}

template <class T>
void upload(DevBuf<T> &b, const std::vector<T> &h) {
    b.alloc(h.size());
    if (!h.empty())
        CH_CUDA_TRY(cudaMemcpy(b.ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
}

// A rank-ordered CSR of n rows and `edges` entries whose targets are ranks.
bool csr_ok(const std::vector<uint32_t> &off, const std::vector<uint2> &adj, uint64_t n) {
    if (off.size() != n + 1 || off[0] != 0 || off[n] != adj.size()) return false;
    for (uint64_t i = 0; i < n; ++i)
        if (off[i] > off[i + 1]) return false;
    for (const uint2 &e : adj)
        if (e.x >= n) return false;
    return true;
}

__global__ void k_fill(uint32_t *a, uint64_t k, uint32_t v) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < k;
         i += (uint64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

}  // namespace

void save_hierarchy(const ch_s *h, const char *path) {
    File file;
    file.f = std::fopen(path, "wb");
    if (!file.f) throw Error{CH_EINVAL, std::string("cannot open for writing: ") + path};
    FileHeader hd{};
    hd.n = h->n;
    hd.hop_limit = h->hop_limit;
    hd.m_input = h->m_input;
    hd.n_up = h->n_up;
    hd.n_down = h->n_down;
    hd.n_shortcuts = h->n_shortcuts;
    hd.rounds = h->round_stats.size();
    hd.core_size = h->core_size;
    hd.nstat = CH_NSTAT;
    hd.ntime = CH_NTIME;
    put(file.f, kMagic, sizeof(kMagic));
    put(file.f, &hd, sizeof(hd));
    const uint64_t n = h->n;
    put_dev(file.f, h->rank, n);
    put_dev(file.f, h->perm, n);
    put_dev(file.f, h->level, n);
    put_dev(file.f, h->prio, n);
    put_dev(file.f, h->up_off, n + 1);
    put_dev(file.f, h->dn_off, n + 1);
    put_dev(file.f, h->up_adj, h->n_up);
    put_dev(file.f, h->dn_adj, h->n_down);
    put_dev(file.f, h->sc, h->n_shortcuts);
    put_dev(file.f, h->sc_round, h->n_shortcuts);
    for (const auto &row : h->round_stats) put(file.f, row.data(), sizeof(row));
    for (const auto &row : h->round_times) put(file.f, row.data(), sizeof(row));
    put(file.f, &h->stats, sizeof(h->stats));
    if (std::fflush(file.f) != 0) throw Error{CH_EINVAL, "write failed"};
}

ch_s *load_hierarchy(const char *path) {
    File file;
    file.f = std::fopen(path, "rb");
    if (!file.f) throw Error{CH_EINVAL, std::string("cannot open for reading: ") + path};
    char magic[8];
    get(file.f, magic, sizeof(magic));
    if (std::memcmp(magic, kMagic, sizeof(magic)) != 0) throw Error{CH_EINVAL, "not a saved hierarchy"};
    FileHeader hd{};
    get(file.f, &hd, sizeof(hd));
    if (hd.nstat != CH_NSTAT || hd.ntime != CH_NTIME || hd.n == 0xFFFFFFFFu || hd.n_up >= 0xFFFFFFFFull ||
        hd.n_down >= 0xFFFFFFFFull || hd.rounds > 0x7FFFFFFFull || hd.n_shortcuts > (1ull << 40))
        throw Error{CH_EINVAL, "saved hierarchy has an unsupported layout"};
    // the sizes the header states must match the file before anything is
    // allocated for them
    const uint64_t n64 = hd.n;
    const uint64_t want = sizeof(kMagic) + sizeof(hd) + 4 * n64 * 4 + 2 * (n64 + 1) * 4 +
                          (hd.n_up + hd.n_down) * sizeof(uint2) + hd.n_shortcuts * (sizeof(uint4) + 4) +
                          hd.rounds * (sizeof(uint64_t) * CH_NSTAT + sizeof(double) * CH_NTIME) +
                          sizeof(ch_stats_t);
    const long here = std::ftell(file.f);
    if (here < 0 || std::fseek(file.f, 0, SEEK_END) != 0) throw Error{CH_EINVAL, "cannot read the file"};
    const long size = std::ftell(file.f);
    if (size < 0 || (uint64_t)size != want || std::fseek(file.f, here, SEEK_SET) != 0)
        throw Error{CH_EINVAL, "file size does not match the saved hierarchy's header"};
    std::unique_ptr<ch_s> h(new (std::nothrow) ch_s());
    if (!h) throw Error{CH_ENOMEM, "host allocation failed"};
    CH_CUDA_TRY(cudaGetDevice(&h->device));
    h->n = hd.n;
    h->hop_limit = hd.hop_limit;
    h->m_input = hd.m_input;
    h->n_up = hd.n_up;
    h->n_down = hd.n_down;
    h->n_shortcuts = hd.n_shortcuts;
    h->core_size = hd.core_size;
    const uint64_t n = hd.n;
    // read everything, check it, then upload: a damaged file must not put
    // out-of-range indices into the hierarchy
    const auto rank = get_vec<uint32_t>(file.f, n);
    const auto perm = get_vec<uint32_t>(file.f, n);
    const auto level = get_vec<uint32_t>(file.f, n);
    const auto prio = get_vec<int32_t>(file.f, n);
    const auto up_off = get_vec<uint32_t>(file.f, n + 1);
    const auto dn_off = get_vec<uint32_t>(file.f, n + 1);
    const auto up_adj = get_vec<uint2>(file.f, hd.n_up);
    const auto dn_adj = get_vec<uint2>(file.f, hd.n_down);
    const auto sc = get_vec<uint4>(file.f, hd.n_shortcuts);
    const auto sc_round = get_vec<uint32_t>(file.f, hd.n_shortcuts);
    h->round_stats.resize(hd.rounds);
    h->round_times.resize(hd.rounds);
    for (auto &row : h->round_stats) get(file.f, row.data(), sizeof(row));
    for (auto &row : h->round_times) get(file.f, row.data(), sizeof(row));
    get(file.f, &h->stats, sizeof(h->stats));
    h->stats.trace_rows = 0;  // traces are not saved
    bool ok = csr_ok(up_off, up_adj, n) && csr_ok(dn_off, dn_adj, n);
    for (uint64_t i = 0; ok && i < n; ++i) ok = rank[i] < n && perm[rank[i]] == i;
    for (uint64_t i = 0; ok && i < hd.n_shortcuts; ++i) ok = sc[i].x < n && sc[i].y < n && sc[i].w < n;
    if (!ok || h->stats.n != hd.n || h->stats.rounds != hd.rounds)
        throw Error{CH_EINVAL, "saved hierarchy is inconsistent"};
    upload(h->rank, rank);
    upload(h->perm, perm);
    upload(h->level, level);
    upload(h->prio, prio);
    upload(h->up_off, up_off);
    upload(h->dn_off, dn_off);
    upload(h->up_adj, up_adj);
    upload(h->dn_adj, dn_adj);
    upload(h->sc, sc);
    upload(h->sc_round, sc_round);
    query_init(h.get());
    return h.release();
}

void query_one_to_many(ch_s *h, uint32_t s, const uint32_t *dst, uint64_t k, uint32_t *dist_out,
                       cudaStream_t st) {
    if (k == 0) return;
    if (h->q_src_fill.count < k) h->q_src_fill.alloc(k);
    k_fill<<<grid_for(k, 256, device_sm_count() * 4), 256, 0, st>>>(h->q_src_fill.ptr, k, s);
    CH_CHECK_LAUNCH();
    query_batch(h, h->q_src_fill.ptr, dst, k, dist_out, nullptr, st);
}

}  // namespace gbch
