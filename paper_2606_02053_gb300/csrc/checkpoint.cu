// Checkpoint / resume of one grid's state (declared in include/cosmos.h).
//
// File layout: a 4096-byte text header, then the payload.  The header is one
// JSON object (the grid sizes, spacing and origin, the field count and names
// in state order, the evolution parameters, the time and step counter, the
// payload's size and FNV-1a 64-bit hash), padded with spaces and ended by a
// newline.  The payload holds every field as nx * ny * nz IEEE binary64
// values in the host's byte order (the header names it), i fastest, field
// after field; padding columns are not stored.  Doubles in the header are
// written with 17 significant digits, so they read back exactly.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "host.cuh"

namespace cosmos {
namespace {

constexpr size_t kHeaderBytes = 4096;
constexpr uint64_t kFnvOffset = 0xcbf29ce484222325ull, kFnvPrime = 0x100000001b3ull;

const char* const kFieldNames[30] = {"chi",   "gt_xx", "gt_xy", "gt_xz", "gt_yy", "gt_yz", "gt_zz", "K",
                                     "At_xx", "At_xy", "At_xz", "At_yy", "At_yz", "At_zz", "Gt_x",  "Gt_y",
                                     "Gt_z",  "alpha", "beta_x", "beta_y", "beta_z", "B_x",  "B_y",   "B_z",
                                     "tau",   "S_x",   "S_y",   "S_z",   "phi",   "Pi"};

int nfields_of(const cosmos_params* p) { return 24 + 4 * p->fluid + 2 * p->scalar; }

// name of state field f (the scalar's two fields follow the fluid's, or the
// vacuum fields when the fluid is off)
const char* field_name(const cosmos_params* p, int f) { return kFieldNames[(!p->fluid && f >= 24) ? f + 4 : f]; }

uint64_t fnv1a(uint64_t h, const unsigned char* b, size_t n) {
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * kFnvPrime;
  return h;
}

bool little_endian() {
  const uint16_t one = 1;
  unsigned char c;
  memcpy(&c, &one, 1);
  return c == 1;
}

void put_d(std::string& s, double v) {
  char b[40];
  snprintf(b, sizeof(b), "%.17g", v);
  s += b;
}

std::string header_json(const cosmos_grid* g, const cosmos_params* p, double t, long long step, uint64_t bytes,
                        uint64_t hash) {
  std::string s = "{\"format\": \"cosmos-checkpoint\", \"version\": 1, \"byte_order\": \"";
  s += little_endian() ? "little" : "big";
  s += "\", \"n\": [" + std::to_string(g->nx) + ", " + std::to_string(g->ny) + ", " + std::to_string(g->nz) + "]";
  s += ", \"h\": [";
  for (int d = 0; d < 3; ++d) {
    if (d) s += ", ";
    put_d(s, g->h[d]);
  }
  s += "], \"x0\": [";
  for (int d = 0; d < 3; ++d) {
    if (d) s += ", ";
    put_d(s, g->x0[d]);
  }
  s += "], \"nfields\": " + std::to_string(nfields_of(p)) + ", \"fields\": [";
  for (int f = 0; f < nfields_of(p); ++f) s += std::string(f ? ", \"" : "\"") + field_name(p, f) + "\"";
  s += "], \"params\": {\"slicing\": " + std::to_string(p->slicing) + ", \"shift\": " + std::to_string(p->shift) +
       ", \"fluid\": " + std::to_string(p->fluid) + ", \"scalar\": " + std::to_string(p->scalar) + ", \"eta\": ";
  put_d(s, p->eta);
  s += ", \"ko_sigma\": ";
  put_d(s, p->ko_sigma);
  s += ", \"w\": ";
  put_d(s, p->w);
  s += ", \"H0\": ";
  put_d(s, p->H0);
  s += ", \"t0\": ";
  put_d(s, p->t0);
  s += "}, \"t\": ";
  put_d(s, t);
  s += ", \"step\": " + std::to_string(step) + ", \"payload_bytes\": " + std::to_string((unsigned long long)bytes);
  char hx[32];
  snprintf(hx, sizeof(hx), "%016llx", (unsigned long long)hash);
  s += ", \"payload_fnv1a64\": \"" + std::string(hx) + "\"}";
  return s;
}

// The numbers following "key": in the header (an array's elements, or one
// value); false when the key is missing or a number does not parse.
bool header_numbers(const char* h, const char* key, double* out, int count) {
  const std::string k = std::string("\"") + key + "\": ";
  const char* p = strstr(h, k.c_str());
  if (!p) return false;
  p += k.size();
  if (*p == '[') ++p;
  for (int i = 0; i < count; ++i) {
    while (*p == ' ' || *p == ',') ++p;
    char* end = nullptr;
    out[i] = strtod(p, &end);
    if (end == p) return false;
    p = end;
  }
  return true;
}

bool header_string(const char* h, const char* key, std::string* out) {
  const std::string k = std::string("\"") + key + "\": \"";
  const char* p = strstr(h, k.c_str());
  if (!p) return false;
  p += k.size();
  const char* e = strchr(p, '"');
  if (!e) return false;
  out->assign(p, e - p);
  return true;
}

// Copies field f between the caller's (pitched) state and a packed buffer.
int copy_field(const cosmos_grid* g, double* state, int on_device, int f, double* packed, bool to_packed,
               cudaStream_t s) {
  const size_t fs = (size_t)g->pitch * g->ny * g->nz;
  const size_t rows = (size_t)g->ny * g->nz;
  double* base = state + f * fs;
  if (on_device) {
    const cudaError_t e =
        to_packed ? cudaMemcpy2DAsync(packed, g->nx * sizeof(double), base, g->pitch * sizeof(double),
                                      g->nx * sizeof(double), rows, cudaMemcpyDeviceToHost, s)
                  : cudaMemcpy2DAsync(base, g->pitch * sizeof(double), packed, g->nx * sizeof(double),
                                      g->nx * sizeof(double), rows, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return COSMOS_ECUDA;
    return COSMOS_OK;
  }
  for (size_t r = 0; r < rows; ++r) {
    if (to_packed)
      memcpy(packed + r * g->nx, base + r * g->pitch, g->nx * sizeof(double));
    else
      memcpy(base + r * g->pitch, packed + r * g->nx, g->nx * sizeof(double));
  }
  return COSMOS_OK;
}

}  // namespace
}  // namespace cosmos

using namespace cosmos;

extern "C" {

int cosmos_checkpoint_save(const char* path, const cosmos_grid* g, const cosmos_params* p, const double* state,
                           int state_on_device, double t, long long step, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!path || !state) return COSMOS_EINVAL;
  const int nf = nfields_of(p);
  const size_t npts = (size_t)g->nx * g->ny * g->nz;
  std::vector<double> buf(npts);
  const std::string tmp = std::string(path) + ".partial";
  FILE* fp = fopen(tmp.c_str(), "wb");
  if (!fp) return COSMOS_EIO;
  std::vector<char> pad(kHeaderBytes, ' ');
  bool ok = fwrite(pad.data(), 1, kHeaderBytes, fp) == kHeaderBytes;  // header written last
  uint64_t hash = kFnvOffset;
  for (int f = 0; f < nf && ok; ++f) {
    e = copy_field(g, const_cast<double*>(state), state_on_device, f, buf.data(), true, (cudaStream_t)stream);
    if (e) {
      fclose(fp);
      remove(tmp.c_str());
      return e;
    }
    hash = fnv1a(hash, (const unsigned char*)buf.data(), npts * sizeof(double));
    ok = fwrite(buf.data(), sizeof(double), npts, fp) == npts;
  }
  const std::string js = header_json(g, p, t, step, (uint64_t)nf * npts * sizeof(double), hash);
  ok = ok && js.size() < kHeaderBytes - 1;
  if (ok) {
    std::string h = js + std::string(kHeaderBytes - 1 - js.size(), ' ') + "\n";
    ok = fseek(fp, 0, SEEK_SET) == 0 && fwrite(h.data(), 1, kHeaderBytes, fp) == kHeaderBytes;
  }
  ok = (fclose(fp) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return COSMOS_EIO;
  }
  return COSMOS_OK;
}

int cosmos_checkpoint_load(const char* path, const cosmos_grid* g, const cosmos_params* p, double* state,
                           int state_on_device, double* t_out, long long* step_out, void* stream) {
  int e = validate(g, p);
  if (e) return e;
  if (!path || !state) return COSMOS_EINVAL;
  FILE* fp = fopen(path, "rb");
  if (!fp) return COSMOS_EIO;
  std::vector<char> h(kHeaderBytes + 1, 0);
  if (fread(h.data(), 1, kHeaderBytes, fp) != kHeaderBytes) {
    fclose(fp);
    return COSMOS_ECHECKPOINT;
  }
  // the header must describe this grid and these parameters exactly
  const int nf = nfields_of(p);
  const size_t npts = (size_t)g->nx * g->ny * g->nz;
  std::string fmt, order, hash_hex;
  double n[3], hh[3], x0[3], nfd, prm[9], t, stp, bytes;
  bool ok = header_string(h.data(), "format", &fmt) && fmt == "cosmos-checkpoint" &&
            header_string(h.data(), "byte_order", &order) && order == (little_endian() ? "little" : "big") &&
            header_numbers(h.data(), "n", n, 3) && header_numbers(h.data(), "h", hh, 3) &&
            header_numbers(h.data(), "x0", x0, 3) && header_numbers(h.data(), "nfields", &nfd, 1) &&
            header_numbers(h.data(), "slicing", prm + 0, 1) && header_numbers(h.data(), "shift", prm + 1, 1) &&
            header_numbers(h.data(), "fluid", prm + 2, 1) && header_numbers(h.data(), "scalar", prm + 3, 1) &&
            header_numbers(h.data(), "eta", prm + 4, 1) && header_numbers(h.data(), "ko_sigma", prm + 5, 1) &&
            header_numbers(h.data(), "w", prm + 6, 1) && header_numbers(h.data(), "H0", prm + 7, 1) &&
            header_numbers(h.data(), "t0", prm + 8, 1) && header_numbers(h.data(), "t", &t, 1) &&
            header_numbers(h.data(), "step", &stp, 1) && header_numbers(h.data(), "payload_bytes", &bytes, 1) &&
            header_string(h.data(), "payload_fnv1a64", &hash_hex);
  ok = ok && n[0] == g->nx && n[1] == g->ny && n[2] == g->nz && nfd == nf;
  for (int d = 0; d < 3 && ok; ++d) ok = hh[d] == g->h[d] && x0[d] == g->x0[d];
  ok = ok && prm[0] == p->slicing && prm[1] == p->shift && prm[2] == p->fluid && prm[3] == p->scalar &&
       prm[4] == p->eta && prm[5] == p->ko_sigma && prm[6] == p->w && prm[7] == p->H0 && prm[8] == p->t0;
  ok = ok && bytes == (double)nf * npts * sizeof(double);
  if (!ok) {
    fclose(fp);
    return COSMOS_ECHECKPOINT;
  }
  // first pass: hash the payload (one field in memory at a time) before
  // touching the caller's state; second pass: copy it in
  std::vector<double> buf(npts);
  uint64_t hash = kFnvOffset;
  bool full = true;
  for (int f = 0; f < nf && full; ++f) {
    full = fread(buf.data(), sizeof(double), npts, fp) == npts;
    hash = fnv1a(hash, (const unsigned char*)buf.data(), npts * sizeof(double));
  }
  const bool at_end = full && fgetc(fp) == EOF;
  char hx[32];
  snprintf(hx, sizeof(hx), "%016llx", (unsigned long long)hash);
  if (!full || !at_end || hash_hex != hx || fseek(fp, (long)kHeaderBytes, SEEK_SET) != 0) {
    fclose(fp);
    return COSMOS_ECHECKPOINT;
  }
  // the second pass is hashed too: a file rewritten or failing between the
  // passes is reported (the state then holds unverified data: COSMOS_EIO)
  uint64_t hash2 = kFnvOffset;
  for (int f = 0; f < nf; ++f) {
    if (fread(buf.data(), sizeof(double), npts, fp) != npts) {
      fclose(fp);
      return COSMOS_EIO;
    }
    hash2 = fnv1a(hash2, (const unsigned char*)buf.data(), npts * sizeof(double));
    e = copy_field(g, state, state_on_device, f, buf.data(), false, (cudaStream_t)stream);
    if (e) {
      fclose(fp);
      return e;
    }
  }
  fclose(fp);
  if (hash2 != hash) return COSMOS_EIO;
  if (t_out) *t_out = t;
  if (step_out) *step_out = (long long)stp;
  return COSMOS_OK;
}

}  // extern "C"
