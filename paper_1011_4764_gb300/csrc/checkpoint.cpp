// Checkpoint of the basis (Sec. II: the fragment eigenstates are computed
// once and then used by every pair): the states of every fragment written
// to <path>.bin as raw little-endian values in the storage precision, one
// fragment after another, each P_a x n_a column-major (state i contiguous,
// box points x fastest, the layout of ofm_get_fragment_states), with a
// JSON header <path>.json that records the geometry they belong to.  A
// later context with the same grid, boxes and state counts resumes from
// them (ofm_load_basis), skipping the eigensolve.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ofm_internal.h"

namespace {

// The header: every field on its own line, so the reader below can check
// the geometry without a general JSON parser.
std::string basis_header(const ofm_ctx* c) {
  std::string h = "{\n";
  char buf[256];
  h += "\"format\": \"ofm-basis-1\",\n";
  snprintf(buf, sizeof buf, "\"grid\": [%d, %d, %d],\n", c->grid.n[0], c->grid.n[1], c->grid.n[2]);
  h += buf;
  snprintf(buf, sizeof buf, "\"h\": %.17g,\n", c->grid.h);
  h += buf;
  h += std::string("\"storage\": \"") + (c->storage == OFM_STORE_FP64 ? "fp64" : "fp32") + "\",\n";
  h += "\"layout\": \"per fragment P_a x n_a column-major, box points x fastest, little-endian\",\n";
  snprintf(buf, sizeof buf, "\"n_frag\": %d,\n", c->nfrag);
  h += buf;
  h += "\"fragments\": [\n";
  for (int a = 0; a < c->nfrag; ++a) {
    const ofm_fragment& f = c->in_frags[a];
    snprintf(buf, sizeof buf, "[%d, %d, %d, %d, %d, %d, %d]%s\n", f.off[0], f.off[1], f.off[2],
             f.ext[0], f.ext[1], f.ext[2], f.n_states, a + 1 < c->nfrag ? "," : "");
    h += buf;
  }
  h += "]\n}\n";
  return h;
}

bool read_file(const std::string& path, std::string& out) {
  FILE* fp = std::fopen(path.c_str(), "rb");
  if (!fp) return false;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, fp)) > 0) out.append(buf, n);
  std::fclose(fp);
  return true;
}

}  // namespace

extern "C" ofm_status ofm_save_basis(ofm_ctx* c, const char* path) {
  if (!c) return OFM_ERR_INVALID;
  OFM_RANGE("ofm_save_basis");
  if (!path) return ofm_fail(c, OFM_ERR_INVALID, "path must not be NULL");
  if (!c->built || !c->have_states) return ofm_fail(c, OFM_ERR_STATE, "no fragment states to save");
  const std::string base(path);
  FILE* fb = std::fopen((base + ".bin").c_str(), "wb");
  if (!fb) return ofm_fail(c, OFM_ERR_INVALID, "cannot open " + base + ".bin for writing");
  std::vector<double> st;
  std::vector<float> st32;
  const bool f64 = c->storage == OFM_STORE_FP64;
  for (int a = 0; a < c->nfrag; ++a) {
    const ofm_fragment& f = c->in_frags[a];
    const size_t cnt = (size_t)f.ext[0] * f.ext[1] * f.ext[2] * f.n_states;
    st.resize(cnt);
    const ofm_status s = ofm_get_fragment_states(c, a, st.data(), OFM_HOST);
    if (s != OFM_OK) {
      std::fclose(fb);
      return s;
    }
    size_t wrote;
    if (f64) {
      wrote = std::fwrite(st.data(), sizeof(double), cnt, fb);
    } else {   // the storage precision: the FP32 values exactly
      st32.resize(cnt);
      for (size_t i = 0; i < cnt; ++i) st32[i] = (float)st[i];
      wrote = std::fwrite(st32.data(), sizeof(float), cnt, fb);
    }
    if (wrote != cnt) {
      std::fclose(fb);
      return ofm_fail(c, OFM_ERR_INVALID, "short write to " + base + ".bin");
    }
  }
  if (std::fclose(fb) != 0) return ofm_fail(c, OFM_ERR_INVALID, "cannot close " + base + ".bin");
  FILE* fh = std::fopen((base + ".json").c_str(), "wb");
  if (!fh) return ofm_fail(c, OFM_ERR_INVALID, "cannot open " + base + ".json for writing");
  const std::string h = basis_header(c);
  const bool ok = std::fwrite(h.data(), 1, h.size(), fh) == h.size();
  if (std::fclose(fh) != 0 || !ok) return ofm_fail(c, OFM_ERR_INVALID, "cannot write " + base + ".json");
  return OFM_OK;
}

extern "C" ofm_status ofm_load_basis(ofm_ctx* c, const char* path) {
  if (!c) return OFM_ERR_INVALID;
  OFM_RANGE("ofm_load_basis");
  if (!path) return ofm_fail(c, OFM_ERR_INVALID, "path must not be NULL");
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  const std::string base(path);
  std::string hdr;
  if (!read_file(base + ".json", hdr)) return ofm_fail(c, OFM_ERR_INVALID, "cannot read " + base + ".json");
  // the saved header must be the one this context would write: the same
  // grid, boxes, state counts and storage
  if (hdr != basis_header(c))
    return ofm_fail(c, OFM_ERR_INVALID,
                    base + ".json: the checkpoint belongs to another grid, box list, state count or storage");
  FILE* fb = std::fopen((base + ".bin").c_str(), "rb");
  if (!fb) return ofm_fail(c, OFM_ERR_INVALID, "cannot open " + base + ".bin");
  const bool f64 = c->storage == OFM_STORE_FP64;
  std::vector<double> st;
  std::vector<float> st32;
  for (int a = 0; a < c->nfrag; ++a) {
    const ofm_fragment& f = c->in_frags[a];
    const size_t cnt = (size_t)f.ext[0] * f.ext[1] * f.ext[2] * f.n_states;
    st.resize(cnt);
    size_t got;
    if (f64) {
      got = std::fread(st.data(), sizeof(double), cnt, fb);
    } else {
      st32.resize(cnt);
      got = std::fread(st32.data(), sizeof(float), cnt, fb);
      for (size_t i = 0; i < got; ++i) st[i] = st32[i];
    }
    if (got != cnt) {
      std::fclose(fb);
      return ofm_fail(c, OFM_ERR_INVALID, base + ".bin is shorter than its header says");
    }
    const ofm_status s = ofm_set_fragment_states(c, a, st.data(), OFM_HOST);
    if (s != OFM_OK) {
      std::fclose(fb);
      return s;
    }
  }
  const bool extra = std::fgetc(fb) != EOF;
  std::fclose(fb);
  if (extra) return ofm_fail(c, OFM_ERR_INVALID, base + ".bin is longer than its header says");
  return OFM_OK;
}
