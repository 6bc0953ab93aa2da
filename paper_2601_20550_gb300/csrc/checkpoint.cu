// Checkpoint files with an integrity check (no counterpart in the paper: the
// resume support a multi-hour c5 run needs).  A file is
//   header  "HEOMCKPT", format version, payload bytes, a 64-byte caller tag
//   payload the caller's bytes
//   trailer CRC-32 (IEEE 802.3 polynomial, reflected, as in zlib) of header and payload
// States are saved as their device storage (complex128 product basis or
// complex64 coupling basis, exactly as held), with their shape in the tag, so a
// load restores them bit for bit.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "internal.h"

namespace heom {
namespace {

constexpr char kMagic[8] = {'H', 'E', 'O', 'M', 'C', 'K', 'P', 'T'};
constexpr uint32_t kVersion = 1;
constexpr size_t kTagBytes = 64;

struct Header {
  char magic[8];
  uint32_t version;
  uint32_t reserved;
  uint64_t payload_bytes;
  unsigned char tag[kTagBytes];
};
static_assert(sizeof(Header) == 88, "checkpoint header layout");

// CRC-32 with the reflected polynomial 0xEDB88320, one table lookup per byte.
struct Crc32 {
  uint32_t table[256];
  Crc32() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? (0xEDB88320u ^ (c >> 1)) : (c >> 1);
      table[i] = c;
    }
  }
  uint32_t update(uint32_t crc, const unsigned char *p, size_t n) const {
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return ~crc;
  }
};

const Crc32 &crc32() {
  static const Crc32 c;
  return c;
}

struct File {
  FILE *f = nullptr;
  explicit File(const char *path, const char *mode) : f(std::fopen(path, mode)) {}
  ~File() {
    if (f) std::fclose(f);
  }
};

void write_file(const char *path, const void *data, uint64_t bytes, const unsigned char *tag) {
  Header h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.payload_bytes = bytes;
  if (tag) std::memcpy(h.tag, tag, kTagBytes);
  uint32_t crc = crc32().update(0, reinterpret_cast<const unsigned char *>(&h), sizeof h);
  crc = crc32().update(crc, static_cast<const unsigned char *>(data), bytes);
  // written to a temporary name and renamed, so an interrupted save leaves the
  // previous checkpoint intact
  const std::string tmp = std::string(path) + ".tmp";
  {
    File f(tmp.c_str(), "wb");
    if (!f.f) throw Fail{HEOM_EINVAL, std::string("cannot open ") + tmp + " for writing"};
    if (std::fwrite(&h, sizeof h, 1, f.f) != 1 || (bytes && std::fwrite(data, 1, bytes, f.f) != bytes) ||
        std::fwrite(&crc, 4, 1, f.f) != 1 || std::fflush(f.f) != 0)
      throw Fail{HEOM_ECKPT, std::string("write failed: ") + tmp};
  }
  if (std::rename(tmp.c_str(), path) != 0) throw Fail{HEOM_ECKPT, std::string("cannot rename to ") + path};
}

// Reads and checks a checkpoint; data may be null (verify only), else it receives
// exactly `bytes` bytes (HEOM_EINVAL if the file holds another size).  on_header
// (may be empty) sees the tag and payload size before the payload is read.
void read_file(const char *path, void *data, uint64_t bytes, uint64_t *size_out,
               const std::function<void(const unsigned char *, uint64_t)> &on_header = {}) {
  File f(path, "rb");
  if (!f.f) throw Fail{HEOM_ECKPT, std::string("cannot open checkpoint ") + path};
  Header h{};
  if (std::fread(&h, sizeof h, 1, f.f) != 1) throw Fail{HEOM_ECKPT, "checkpoint header truncated"};
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion)
    throw Fail{HEOM_ECKPT, "not a checkpoint of this format"};
  if (size_out) *size_out = h.payload_bytes;
  if (on_header) on_header(h.tag, h.payload_bytes);
  if (data && h.payload_bytes != bytes)
    throw Fail{HEOM_EINVAL, "checkpoint holds " + std::to_string(h.payload_bytes) + " bytes, " +
                                std::to_string(bytes) + " expected"};
  uint32_t crc = crc32().update(0, reinterpret_cast<const unsigned char *>(&h), sizeof h);
  std::vector<unsigned char> chunk(data ? 0 : (1u << 20));
  uint64_t left = h.payload_bytes;
  unsigned char *dst = static_cast<unsigned char *>(data);
  while (left > 0) {
    const size_t n = (size_t)std::min<uint64_t>(left, 1u << 20);
    unsigned char *buf = dst ? dst : chunk.data();
    if (std::fread(buf, 1, n, f.f) != n) throw Fail{HEOM_ECKPT, "checkpoint payload truncated"};
    crc = crc32().update(crc, buf, n);
    if (dst) dst += n;
    left -= n;
  }
  uint32_t stored = 0;
  if (std::fread(&stored, 4, 1, f.f) != 1) throw Fail{HEOM_ECKPT, "checkpoint trailer truncated"};
  if (stored != crc) throw Fail{HEOM_ECKPT, "checkpoint CRC mismatch"};
}

// Tag of a saved state: its shape and representation.
struct StateTag {
  int32_t branches, precision, d, n_ado;
  int64_t eq_steps;
  double eq_dt;
};
static_assert(sizeof(StateTag) <= kTagBytes, "state tag fits the header");

}  // namespace
}  // namespace heom

extern "C" {

heom_status heom_ckpt_write(const char *path, const void *host, uint64_t bytes) {
  if (!path || (!host && bytes)) return fail(HEOM_EINVAL, "bad checkpoint arguments");
  return guarded([&]() -> heom_status {
    write_file(path, host, bytes, nullptr);
    return HEOM_OK;
  });
}

heom_status heom_ckpt_read(const char *path, void *host, uint64_t bytes) {
  if (!path || (!host && bytes)) return fail(HEOM_EINVAL, "bad checkpoint arguments");
  return guarded([&]() -> heom_status {
    std::vector<unsigned char> tmp(bytes);
    read_file(path, tmp.data(), bytes, nullptr);
    if (bytes) std::memcpy(host, tmp.data(), bytes);   // the caller's buffer changes only on success
    return HEOM_OK;
  });
}

heom_status heom_ckpt_verify(const char *path, uint64_t *payload_bytes) {
  if (!path) return fail(HEOM_EINVAL, "null path");
  return guarded([&]() -> heom_status {
    read_file(path, nullptr, 0, payload_bytes);
    return HEOM_OK;
  });
}

heom_status heom_state_save(const heom_state *s, const char *path) {
  if (!s || !path) return fail(HEOM_EINVAL, "null argument");
  return guarded([&]() -> heom_status {
    const uint64_t bytes = (uint64_t)s->elems() * s->elem_bytes();
    std::vector<unsigned char> host(bytes);
    CUDA_TRY(cudaDeviceSynchronize());   // work on any stream that writes the state is done
    CUDA_TRY(cudaMemcpy(host.data(), s->buf.p, bytes, cudaMemcpyDeviceToHost));
    unsigned char tag[kTagBytes] = {0};
    StateTag t{s->branches, s->precision, s->d, s->n_ado, s->eq_steps, s->eq_dt};
    std::memcpy(tag, &t, sizeof t);
    write_file(path, host.data(), bytes, tag);
    return HEOM_OK;
  });
}

heom_status heom_state_load(heom_state *s, const char *path) {
  if (!s || !path) return fail(HEOM_EINVAL, "null argument");
  return guarded([&]() -> heom_status {
    const uint64_t bytes = (uint64_t)s->elems() * s->elem_bytes();
    std::vector<unsigned char> host(bytes);
    StateTag t{};
    read_file(path, host.data(), bytes, nullptr, [&](const unsigned char *tag, uint64_t) {
      std::memcpy(&t, tag, sizeof t);
      if (t.branches != s->branches || t.precision != s->precision || t.d != s->d || t.n_ado != s->n_ado)
        throw Fail{HEOM_EINVAL, "checkpoint holds a state of another shape or precision"};
    });
    // the device state changes only once the whole file has passed its check
    CUDA_TRY(cudaMemcpy(s->buf.p, host.data(), bytes, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaDeviceSynchronize());   // complete before work on any stream reads it
    s->eq_steps = t.eq_steps;
    s->eq_dt = t.eq_dt;
    return HEOM_OK;
  });
}

}  // extern "C"
