// files.cpp -- PDB table files: a fixed header (pattern, sizes, hash) and the table bytes, so
// that tables built once (breadth-first search over the abstract space, Background: PDBs) can
// be reused.  Host code only.
#include <cerrno>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "../../include/cbdfs.h"

namespace cbdfs {

int fail(int code, const char *fmt, ...);

// FNV-1a, 64 bits (offset basis 14695981039346656037, prime 1099511628211), continued from h
uint64_t fnv1a64(const void *data, size_t n, uint64_t h) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}
constexpr uint64_t kFnvBasis = 14695981039346656037ull;

namespace {

struct PdbFileHeader {
    char magic[8];
    uint32_t version;
    int32_t domain, k;
    int32_t tiles[16];
    uint32_t div;
    uint64_t entries;
    uint64_t hash;
    unsigned char pad[128 - 8 - 4 - 8 - 64 - 4 - 8 - 8];
};
static_assert(sizeof(PdbFileHeader) == 128, "the PDB file header is 128 bytes");
constexpr char kPdbMagic[8] = {'C', 'B', 'D', 'F', 'S', 'P', 'D', 'B'};

// entries of a table for (domain, k, div): sliding-tile patterns of k tiles have
// N!/(N-k)! ranks (N = 9 or 16 cells, k <= N-1); the cube's table is the 8-corner one, 8! 3^7
// entries; DIV compression keeps ceil(ranks / div).  0 when the pattern is not one of these.
uint64_t table_entries(int domain, int k, uint32_t div) {
    if (div < 1) return 0;
    uint64_t ranks = 0;
    if (domain == CBDFS_DOM_STP3 || domain == CBDFS_DOM_STP4) {
        const int N = domain == CBDFS_DOM_STP3 ? 9 : 16;
        if (k < 1 || k > N - 1) return 0;
        ranks = 1;
        for (int i = 0; i < k; ++i) ranks *= (uint64_t)(N - i);
    } else if (domain == CBDFS_DOM_RC3) {
        if (k != 8) return 0;
        ranks = 40320ull * 2187ull;
    } else {
        return 0;
    }
    return (ranks + div - 1) / div;
}

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

}  // namespace

}  // namespace cbdfs

using namespace cbdfs;

extern "C" {

int cbdfs_pdb_file_write(const char *path, int domain, const int *tiles, int k, uint32_t div,
                         const uint8_t *table, uint64_t entries) {
    if (!path || !tiles || (!table && entries)) return fail(CBDFS_EINVAL, "null argument");
    if (domain < 0 || domain > 2 || k < 1 || k > 16 || div < 1) return fail(CBDFS_EINVAL, "pattern");
    if (entries != table_entries(domain, k, div))
        return fail(CBDFS_EINVAL, "%llu entries; a table of %d tiles (domain %d, DIV %u) has %llu",
                    (unsigned long long)entries, k, domain, div,
                    (unsigned long long)table_entries(domain, k, div));
    PdbFileHeader hd;
    std::memset(&hd, 0, sizeof hd);
    std::memcpy(hd.magic, kPdbMagic, 8);
    hd.version = 1;
    hd.domain = domain;
    hd.k = k;
    for (int i = 0; i < k; ++i) hd.tiles[i] = tiles[i];
    hd.div = div;
    hd.entries = entries;
    hd.hash = fnv1a64(table, entries, kFnvBasis);
    File out;
    out.f = fopen(path, "wb");
    if (!out.f) return fail(CBDFS_EDEVICE, "%s: %s", path, strerror(errno));
    if (fwrite(&hd, sizeof hd, 1, out.f) != 1 || (entries && fwrite(table, 1, entries, out.f) != entries))
        return fail(CBDFS_EDEVICE, "%s: short write", path);
    if (fclose(out.f) != 0) {
        out.f = nullptr;
        return fail(CBDFS_EDEVICE, "%s: close", path);
    }
    out.f = nullptr;
    return CBDFS_OK;
}

int cbdfs_pdb_file_read(const char *path, int *domain, int *tiles, int *k, uint32_t *div,
                        uint8_t *table, uint64_t cap, uint64_t *entries) {
    if (!path || !domain || !tiles || !k || !div || !entries) return fail(CBDFS_EINVAL, "null argument");
    File in;
    in.f = fopen(path, "rb");
    if (!in.f) return fail(CBDFS_ENOTFOUND, "%s: %s", path, strerror(errno));
    PdbFileHeader hd;
    if (fread(&hd, sizeof hd, 1, in.f) != 1 || std::memcmp(hd.magic, kPdbMagic, 8) != 0)
        return fail(CBDFS_EINVAL, "%s is not a PDB file", path);
    if (hd.version != 1) return fail(CBDFS_EINVAL, "%s: format version %u", path, hd.version);
    if (hd.k < 1 || hd.k > 16) return fail(CBDFS_EINVAL, "%s: pattern size %d", path, hd.k);
    if (hd.domain < 0 || hd.domain > 2) return fail(CBDFS_EINVAL, "%s: domain %d", path, hd.domain);
    if (hd.div < 1) return fail(CBDFS_EINVAL, "%s: DIV factor %u", path, hd.div);
    if (hd.entries != table_entries(hd.domain, hd.k, hd.div))
        return fail(CBDFS_EINVAL, "%s: %llu entries, but a table of %d tiles (domain %d, DIV %u) has %llu", path,
                    (unsigned long long)hd.entries, hd.k, hd.domain, hd.div,
                    (unsigned long long)table_entries(hd.domain, hd.k, hd.div));
    *domain = hd.domain;
    *k = hd.k;
    for (int i = 0; i < 16; ++i) tiles[i] = hd.tiles[i];
    *div = hd.div;
    *entries = hd.entries;
    if (!table) return CBDFS_OK;
    if (cap < hd.entries) return fail(CBDFS_EINVAL, "%s: %llu entries, room for %llu", path,
                                      (unsigned long long)hd.entries, (unsigned long long)cap);
    if (hd.entries && fread(table, 1, hd.entries, in.f) != hd.entries) return fail(CBDFS_EINVAL, "%s: short file", path);
    if (fnv1a64(table, hd.entries, kFnvBasis) != hd.hash) return fail(CBDFS_EINVAL, "%s: hash mismatch", path);
    return CBDFS_OK;
}

}  // extern "C"
