// Index files: a codes handle (PEOs codes or SimHash bits) saved to disk and loaded back,
// so an index is built once and searched across processes.
//
// Layout (little-endian):
//   header   "PEOSIDX1", u32 version, u32 kind, i64 n, i32 R, L, m, d, entry, u64 seed,
//            u64 record stride, i32 node-table stride, i32 scalar width, u32 section count
//   table    per section: u32 id, u32 CRC-32 of its bytes, u64 byte count
//   u32      CRC-32 of the header and the table
//   sections in table order: records, node tables, A, B, Wt, permutation, row norms
//            (the ones the handle has)
// CRC-32 is the IEEE 802.3 / zlib polynomial (reflected 0xEDB88320).  Sections move
// between the device and the file in chunks of at most 64 MiB of host memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace peos {
namespace {

constexpr char kMagic[8] = {'P', 'E', 'O', 'S', 'I', 'D', 'X', '1'};
constexpr uint32_t kVersion = 4;
constexpr size_t kChunk = (size_t)64 << 20;
enum : uint32_t { kSecRecords = 1, kSecNodeTab, kSecA, kSecB, kSecWt, kSecPerm, kSecNorms, kSecCount };

uint32_t crc_table[256];
std::once_flag crc_once;

void crc_init() {
  std::call_once(crc_once, [] {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? (0xEDB88320u ^ (c >> 1)) : (c >> 1);
      crc_table[i] = c;
    }
  });
}

// running CRC: start with 0xFFFFFFFF, finish with ^ 0xFFFFFFFF
uint32_t crc_update(uint32_t crc, const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) crc = crc_table[(crc ^ p[i]) & 0xffu] ^ (crc >> 8);
  return crc;
}

#pragma pack(push, 1)
struct Header {
  char magic[8];
  uint32_t version, kind;
  int64_t n;
  int32_t R, L, m, d, entry;
  uint64_t seed, rec_stride;
  int32_t node_stride;
  int32_t scalar_bits;
  uint32_t nsec;
};
struct SecEntry {
  uint32_t id, crc;
  uint64_t bytes;
};
#pragma pack(pop)

struct Section {
  uint32_t id;
  void* dev;        // device array (owned by the handle)
  uint64_t bytes;
};

std::vector<Section> sections_of(const peos_codes_s* c) {
  const uint64_t n = (uint64_t)c->n;
  const uint64_t md4 = (uint64_t)c->m * c->d * 4;
  std::vector<Section> v;
  v.push_back({kSecRecords, c->records, n * c->rec_stride});
  v.push_back({kSecNodeTab, c->node_proj, n * (uint64_t)node_table_stride(c) * 4});
  if (c->A) v.push_back({kSecA, c->A, md4});
  v.push_back({kSecB, c->B, md4});
  if (c->Wt) v.push_back({kSecWt, c->Wt, 2 * md4});
  if (c->perm) v.push_back({kSecPerm, c->perm, (uint64_t)c->d * 4});
  if (c->norms) v.push_back({kSecNorms, c->norms, n * 4});
  return v;
}

// chunked device -> file copy of one section, returning its CRC
bool write_section(FILE* f, const Section& sec, std::vector<unsigned char>& buf, uint32_t* crc_out) {
  uint32_t crc = 0xFFFFFFFFu;
  for (uint64_t off = 0; off < sec.bytes; off += kChunk) {
    const size_t len = (size_t)std::min<uint64_t>(kChunk, sec.bytes - off);
    if (cudaMemcpy(buf.data(), static_cast<const unsigned char*>(sec.dev) + off, len, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return false;
    crc = crc_update(crc, buf.data(), len);
    if (fwrite(buf.data(), 1, len, f) != len) return false;
  }
  *crc_out = crc ^ 0xFFFFFFFFu;
  return true;
}

bool read_section(FILE* f, void* dev, uint64_t bytes, std::vector<unsigned char>& buf, uint32_t* crc_out) {
  uint32_t crc = 0xFFFFFFFFu;
  for (uint64_t off = 0; off < bytes; off += kChunk) {
    const size_t len = (size_t)std::min<uint64_t>(kChunk, bytes - off);
    if (fread(buf.data(), 1, len, f) != len) return false;
    crc = crc_update(crc, buf.data(), len);
    if (cudaMemcpy(static_cast<unsigned char*>(dev) + off, buf.data(), len, cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
  }
  *crc_out = crc ^ 0xFFFFFFFFu;
  return true;
}

}  // namespace
}  // namespace peos

using namespace peos;

extern "C" {

peos_status peos_crc32(const void* data, size_t bytes, uint32_t* out) {
  if (!out || (!data && bytes)) return set_error(PEOS_E_INVAL, "NULL argument");
  crc_init();
  *out = crc_update(0xFFFFFFFFu, data, bytes) ^ 0xFFFFFFFFu;
  return PEOS_OK;
}

peos_status peos_codes_save(peos_codes_t c, const char* path) {
  if (!c || !path) return set_error(PEOS_E_INVAL, "NULL argument");
  crc_init();
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaSetDevice(cur);
    return cuda_error(e, "peos_codes_save");
  }
  const std::vector<Section> secs = sections_of(c);
  Header h;
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.kind = (uint32_t)c->kind;
  h.n = c->n;
  h.R = c->R;
  h.L = c->L;
  h.m = c->m;
  h.d = c->d;
  h.entry = c->entry;
  h.seed = c->seed;
  h.rec_stride = c->rec_stride;
  h.node_stride = node_table_stride(c);
  h.scalar_bits = c->scalar_bits;
  h.nsec = (uint32_t)secs.size();
  std::vector<SecEntry> table(secs.size());
  FILE* f = fopen(path, "wb");
  if (!f) {
    cudaSetDevice(cur);
    return set_error(PEOS_E_INVAL, std::string("cannot open ") + path + " for writing");
  }
  std::vector<unsigned char> buf;
  bool ok = true;
  try {
    buf.resize(kChunk);
  } catch (...) {
    ok = false;
  }
  // header and table are written twice: placeholders first, the CRCs once known
  const long table_end = (long)(sizeof(Header) + table.size() * sizeof(SecEntry) + sizeof(uint32_t));
  ok = ok && fseek(f, table_end, SEEK_SET) == 0;
  for (size_t i = 0; ok && i < secs.size(); ++i) {
    table[i].id = secs[i].id;
    table[i].bytes = secs[i].bytes;
    ok = write_section(f, secs[i], buf, &table[i].crc);
  }
  if (ok) {
    uint32_t hc = crc_update(0xFFFFFFFFu, &h, sizeof(h));
    hc = crc_update(hc, table.data(), table.size() * sizeof(SecEntry)) ^ 0xFFFFFFFFu;
    ok = fseek(f, 0, SEEK_SET) == 0 && fwrite(&h, sizeof(h), 1, f) == 1 &&
         (table.empty() || fwrite(table.data(), sizeof(SecEntry), table.size(), f) == table.size()) &&
         fwrite(&hc, sizeof(hc), 1, f) == 1;
  }
  ok = (fclose(f) == 0) && ok;
  cudaSetDevice(cur);
  if (!ok) return set_error(PEOS_E_INVAL, std::string("writing ") + path + " failed");
  return PEOS_OK;
}

peos_status peos_codes_graph(peos_codes_t c, int32_t* nbrs, int32_t* entry, void* stream) {
  if (!c || !entry || (c->n > 0 && !nbrs)) return set_error(PEOS_E_INVAL, "NULL argument");
  *entry = c->entry;
  if (c->n == 0) return PEOS_OK;
  // the ids of a node's edges sit at rec_ids_offset(R, scalar width) of its record
  const size_t row = (size_t)c->R * sizeof(int32_t);
  const size_t off = rec_ids_offset(c->R, c->kind == kCodesPeos ? c->scalar_bits : 32);
  cudaError_t e = cudaMemcpy2DAsync(nbrs, row, c->records + off, c->rec_stride, row, (size_t)c->n,
                                    cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "peos_codes_graph");
  return PEOS_OK;
}

peos_status peos_codes_load(const char* path, peos_codes_t* out) {
  if (!path || !out) return set_error(PEOS_E_INVAL, "NULL argument");
  *out = nullptr;
  crc_init();
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(PEOS_E_INVAL, std::string("cannot open ") + path);
  auto bad = [&](const std::string& why, peos_status code = PEOS_E_INVAL) {
    fclose(f);
    return set_error(code, std::string(path) + ": " + why);
  };
  Header h;
  if (fread(&h, sizeof(h), 1, f) != 1) return bad("truncated header");
  if (std::memcmp(h.magic, kMagic, 8) != 0) return bad("not a PEOs index file");
  if (h.version != kVersion) return bad("unsupported version");
  if (h.nsec == 0 || h.nsec >= kSecCount) return bad("bad section count");
  std::vector<SecEntry> table(h.nsec);
  uint32_t hc_file = 0;
  if (fread(table.data(), sizeof(SecEntry), h.nsec, f) != h.nsec || fread(&hc_file, sizeof(hc_file), 1, f) != 1)
    return bad("truncated section table");
  uint32_t hc = crc_update(0xFFFFFFFFu, &h, sizeof(h));
  hc = crc_update(hc, table.data(), table.size() * sizeof(SecEntry)) ^ 0xFFFFFFFFu;
  if (hc != hc_file) return bad("header checksum mismatch");
  // the shape must be one the library builds
  const bool simhash = h.kind == (uint32_t)kCodesSimHash;
  if (h.kind != (uint32_t)kCodesPeos && !simhash) return bad("unknown kind");
  // n is bounded so that no section size below can overflow 64 bits
  if (h.n < 0 || h.n > ((int64_t)1 << 40) || h.R < 1 || h.R > kMaxR || h.L < 1 || h.d < 1 || h.d > (1 << 20) ||
      h.d % h.L != 0 || h.d % 4 != 0 ||
      (h.n > 0 && (h.entry < 0 || h.entry >= h.n)))
    return bad("bad shape");
  if (simhash ? (h.L != 1 || h.m < 64 || h.m > kMaxSimHashBits || h.m % 64 != 0)
              : (h.m < 2 || h.m > 127 || code_words(h.L, h.m) > kMaxCodeWords))
    return bad("bad L / m");
  if (h.scalar_bits != 32 && (simhash || (h.scalar_bits != 16 && h.scalar_bits != 8))) return bad("bad scalar width");
  const uint64_t want_rec =
      simhash ? record_stride_words(h.R, h.m / 64) : record_stride(h.R, h.L, h.m, h.scalar_bits);
  const int want_node = simhash ? h.m : table_stride(h.L, h.m);
  if (h.rec_stride != want_rec || h.node_stride != want_node) return bad("bad strides");

  peos_codes_s* c = new (std::nothrow) peos_codes_s();
  if (!c) return bad("host allocation");
  cudaGetDevice(&c->device);
  c->kind = (int)h.kind;
  c->n = h.n;
  c->R = h.R;
  c->L = h.L;
  c->m = h.m;
  c->d = h.d;
  c->entry = h.entry;
  c->seed = h.seed;
  c->rec_stride = h.rec_stride;
  c->scalar_bits = h.scalar_bits;
  auto release = [&]() {
    cudaFree(c->records);
    cudaFree(c->node_proj);
    cudaFree(c->A);
    cudaFree(c->B);
    cudaFree(c->Wt);
    cudaFree(c->perm);
    cudaFree(c->norms);
    delete c;
  };
  const uint64_t n = (uint64_t)h.n, md4 = (uint64_t)h.m * h.d * 4;
  std::vector<unsigned char> buf;
  try {
    buf.resize(kChunk);
  } catch (...) {
    release();
    return bad("host allocation", PEOS_E_NOMEM);
  }
  uint32_t seen = 0;
  for (const SecEntry& t : table) {
    void** dst = nullptr;
    uint64_t expect = 0;
    switch (t.id) {
      case kSecRecords: dst = reinterpret_cast<void**>(&c->records); expect = n * h.rec_stride; break;
      case kSecNodeTab: dst = reinterpret_cast<void**>(&c->node_proj); expect = n * (uint64_t)want_node * 4; break;
      case kSecA: dst = reinterpret_cast<void**>(&c->A); expect = md4; break;
      case kSecB: dst = reinterpret_cast<void**>(&c->B); expect = md4; break;
      case kSecWt: dst = reinterpret_cast<void**>(&c->Wt); expect = 2 * md4; break;
      case kSecPerm: dst = reinterpret_cast<void**>(&c->perm); expect = (uint64_t)h.d * 4; break;
      case kSecNorms: dst = reinterpret_cast<void**>(&c->norms); expect = n * 4; break;
      default: release(); return bad("unknown section");
    }
    if ((seen >> t.id) & 1u) {
      release();
      return bad("repeated section");
    }
    seen |= 1u << t.id;
    if (t.bytes != expect) {
      release();
      return bad("section size does not match the shape");
    }
    if (cudaMalloc(dst, expect > 0 ? expect : 1) != cudaSuccess) {
      release();
      return bad("device allocation", PEOS_E_NOMEM);
    }
    uint32_t crc = 0;
    if (!read_section(f, *dst, expect, buf, &crc)) {
      release();
      return bad("truncated or unreadable section");
    }
    if (crc != t.crc) {
      release();
      return bad("section checksum mismatch");
    }
    if (t.id == kSecPerm) {  // the search indexes shared memory with it: a permutation of 0..d-1
      std::vector<char> hit(h.d, 0);
      const int32_t* p = reinterpret_cast<const int32_t*>(buf.data());
      for (int i = 0; i < h.d; ++i) {
        if (p[i] < 0 || p[i] >= h.d || hit[p[i]]) {
          release();
          return bad("the permutation section is not a permutation");
        }
        hit[p[i]] = 1;
      }
    }
  }
  const uint32_t need = simhash ? ((1u << kSecRecords) | (1u << kSecNodeTab) | (1u << kSecB))
                                : ((1u << kSecRecords) | (1u << kSecNodeTab) | (1u << kSecA) | (1u << kSecB) |
                                   (1u << kSecWt) | (1u << kSecNorms));
  const uint32_t allowed = need | (simhash || h.scalar_bits != 32 ? 0u : (1u << kSecPerm));
  if ((seen & need) != need || (seen & ~allowed) != 0) {
    release();
    return bad("sections do not match the kind");
  }
  fclose(f);
  if (peos_status r = attach_wide_flags(c, nullptr)) {  // derived from the records: not stored
    release();
    return r;
  }
  *out = c;
  return PEOS_OK;
}

}  // extern "C"
