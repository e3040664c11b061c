// Checkpoint and resume of a CTM environment (host code only).
//
// The CTM state that a move updates is the environment: four corner matrices
// C1..C4 and four edge tensors T1..T4 per cell position.  A checkpoint file
// holds them in the layout ipeps_ctm_env_get returns, behind a small header
// (geometry, so that a load can refuse an environment of another size) and
// followed by a checksum, so that a short or damaged file is refused before
// the handle is touched.  The format is spelled out beside the declarations
// of ipeps_ctm_save / ipeps_ctm_load.
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/ipeps_ctm.h"

#if defined(__BYTE_ORDER__) && __BYTE_ORDER__ != __ORDER_LITTLE_ENDIAN__
#error "the checkpoint format is little-endian; this host is not"
#endif

void set_last_error_message(const char* msg);
void ctm_geometry(ipeps_ctm h, int g[10]);

namespace {

constexpr char kMagic[8] = {'I', 'P', 'E', 'P', 'S', 'E', 'N', 'V'};
constexpr int kVersion = 1;
constexpr int kHeaderInts = 12;  // version, Lx, Ly, d, D, chi, n_tensors, pattern[4], 0
constexpr long kHeaderBytes = 8 + 4 * kHeaderInts;

ipeps_status cfail(ipeps_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error_message(buf);
  return st;
}

// FNV-1a (Fowler, Noll, Vo) with 64-bit words in place of bytes
struct Fnv64 {
  uint64_t h = 0xcbf29ce484222325ULL;
  void words(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i) {
      uint64_t w;
      memcpy(&w, p + i, 8);
      h = (h ^ w) * 0x100000001b3ULL;
    }
  }
};

// complex elements of the environment of one cell position
long long site_elems(int chi, int D) { return 4LL * chi * chi + 4LL * chi * D * D * chi; }

long long role_elems(int role, int chi, int D) {
  return role < 4 ? (long long)chi * chi : (long long)chi * D * D * chi;
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

// Read a checkpoint, check its header, size and checksum.  hdr gets the
// twelve header ints, payload the tensors as doubles.
ipeps_status read_checkpoint(const char* path, int hdr[kHeaderInts], std::vector<double>& payload) {
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) return cfail(IPEPS_EIO, "cannot open %s", path);
  char magic[8];
  if (fread(magic, 1, 8, in.f) != 8 || memcmp(magic, kMagic, 8) != 0)
    return cfail(IPEPS_EIO, "%s is not an environment checkpoint", path);
  if (fread(hdr, 4, kHeaderInts, in.f) != (size_t)kHeaderInts) return cfail(IPEPS_EIO, "%s: short header", path);
  if (hdr[0] != kVersion) return cfail(IPEPS_EIO, "%s: format version %d, expected %d", path, hdr[0], kVersion);
  const int Lx = hdr[1], Ly = hdr[2], D = hdr[4], chi = hdr[5];
  if (Lx < 1 || Lx > 2 || Ly < 1 || Ly > 2 || D < 1 || D > 12 || chi < 1 || chi > 1024)
    return cfail(IPEPS_EIO, "%s: header out of range (Lx %d, Ly %d, D %d, chi %d)", path, Lx, Ly, D, chi);
  const long long n_doubles = 2 * (long long)Lx * Ly * site_elems(chi, D);
  if (fseek(in.f, 0, SEEK_END) != 0) return cfail(IPEPS_EIO, "%s: cannot seek", path);
  const long size = ftell(in.f);
  const long expect = kHeaderBytes + 8 * (long)n_doubles + 8;
  if (size != expect) return cfail(IPEPS_EIO, "%s: %ld bytes, expected %ld", path, size, expect);
  payload.resize((size_t)n_doubles);
  if (fseek(in.f, kHeaderBytes, SEEK_SET) != 0 ||
      fread(payload.data(), 8, (size_t)n_doubles, in.f) != (size_t)n_doubles)
    return cfail(IPEPS_EIO, "%s: short payload", path);
  uint64_t stored;
  if (fread(&stored, 8, 1, in.f) != 1) return cfail(IPEPS_EIO, "%s: missing checksum", path);
  Fnv64 sum;
  sum.words(payload.data(), payload.size());
  if (sum.h != stored) return cfail(IPEPS_EIO, "%s: checksum mismatch (damaged file)", path);
  return IPEPS_OK;
}

}  // namespace

extern "C" ipeps_status ipeps_ctm_save(ipeps_ctm h, const char* path) {
  if (!h || !path) return cfail(IPEPS_EINVAL, "null argument");
  int g[10];
  ctm_geometry(h, g);
  const int Lx = g[0], Ly = g[1], D = g[3], chi = g[4];
  const int hdr[kHeaderInts] = {kVersion, Lx, Ly, g[2], D, chi, g[5], g[6], g[7], g[8], g[9], 0};
  // stage every tensor on the host first: a device error leaves no file behind
  std::vector<double> payload(2 * (size_t)(Lx * Ly * site_elems(chi, D)));
  size_t off = 0;
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x)
      for (int role = 0; role < 8; ++role) {
        ipeps_status st = ipeps_ctm_env_get(h, role, x, y, payload.data() + off);
        if (st != IPEPS_OK) return st;
        off += 2 * (size_t)role_elems(role, chi, D);
      }
  Fnv64 sum;
  sum.words(payload.data(), payload.size());
  const std::string part = std::string(path) + ".part";
  {
    File out;
    out.f = fopen(part.c_str(), "wb");
    if (!out.f) return cfail(IPEPS_EIO, "cannot create %s", part.c_str());
    const bool ok = fwrite(kMagic, 1, 8, out.f) == 8 && fwrite(hdr, 4, kHeaderInts, out.f) == (size_t)kHeaderInts &&
                    fwrite(payload.data(), 8, payload.size(), out.f) == payload.size() &&
                    fwrite(&sum.h, 8, 1, out.f) == 1 && fflush(out.f) == 0;
    const bool closed = fclose(out.f) == 0;
    out.f = nullptr;
    if (!ok || !closed) {
      remove(part.c_str());
      return cfail(IPEPS_EIO, "write to %s failed", part.c_str());
    }
  }
  if (rename(part.c_str(), path) != 0) {
    remove(part.c_str());
    return cfail(IPEPS_EIO, "cannot rename %s to %s", part.c_str(), path);
  }
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_ctm_load(ipeps_ctm h, const char* path) {
  if (!h || !path) return cfail(IPEPS_EINVAL, "null argument");
  int hdr[kHeaderInts];
  std::vector<double> payload;
  ipeps_status st = read_checkpoint(path, hdr, payload);
  if (st != IPEPS_OK) return st;
  int g[10];
  ctm_geometry(h, g);
  const int Lx = g[0], Ly = g[1], D = g[3], chi = g[4];
  if (hdr[1] != Lx || hdr[2] != Ly || hdr[4] != D || hdr[5] != chi)
    return cfail(IPEPS_EINVAL, "%s holds Lx %d, Ly %d, D %d, chi %d; the handle has Lx %d, Ly %d, D %d, chi %d", path,
                 hdr[1], hdr[2], hdr[4], hdr[5], Lx, Ly, D, chi);
  size_t off = 0;
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x)
      for (int role = 0; role < 8; ++role) {
        st = ipeps_ctm_env_set(h, role, x, y, payload.data() + off);
        if (st != IPEPS_OK) return st;
        off += 2 * (size_t)role_elems(role, chi, D);
      }
  return IPEPS_OK;
}

extern "C" ipeps_status ipeps_env_file_info(const char* path, int* info) {
  if (!path || !info) return cfail(IPEPS_EINVAL, "null argument");
  int hdr[kHeaderInts];
  std::vector<double> payload;  // read only to verify the checksum
  ipeps_status st = read_checkpoint(path, hdr, payload);
  if (st != IPEPS_OK) return st;
  for (int i = 0; i < 11; ++i) info[i] = hdr[i];
  return IPEPS_OK;
}
