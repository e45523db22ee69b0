// Checkpoint / resume of the hierarchy and growth of the vertex set.
//
// The maintained hierarchy is the state a batch update resumes from
// (Sec. III-A): every level's graph, parent map, labels, strengths and node
// existence, plus the community totals.  A host image holds exactly that; it
// is written to / read from a file (ldl_save / ldl_load), and the vertex set
// grows (Sec. II: V_t may change) by appending isolated vertices to the image
// and loading it back into the same context (ldl_grow).  Loading builds every
// slack CSR from the image's sorted rows; no static Leiden run is repeated, so
// a loaded context continues exactly where the saved one stood.
#include <cstdio>
#include <cstring>
#include <vector>

#include "kern.cuh"

namespace {

struct LevelImage {
  std::vector<int32_t> lab, par, cnt;
  std::vector<int64_t> kout, kin;  // kin empty when undirected
  std::vector<uint8_t> alive;
  std::vector<int64_t> rp;         // adjacency rows (directed: in-rows after the n out-rows)
  std::vector<int32_t> col;
  std::vector<int64_t> w;
  std::vector<int64_t> crp;        // children lists (levels below the top)
  std::vector<int32_t> ccol;
};

struct Image {
  ldl_params prm{};
  int64_t n = 0;
  int32_t T = 0;
  int64_t m = 0, E = 0;
  int64_t P_hi = 0;
  uint64_t P_lo = 0;
  std::vector<int64_t> Kout, Kin, e;
  std::vector<LevelImage> lv;
};

template <class T>
void dl(ldl_ctx& c, std::vector<T>& dst, const T* src, size_t count) {
  dst.resize(count);
  if (count) CK(cudaMemcpyAsync(dst.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost, c.s));
}

// Rows of a slack CSR as compact sorted rows (rows are kept sorted on the device).
template <class WT>
void csr_rows(ldl_ctx& c, const SlackCSR<WT>& g, int64_t rows, std::vector<int64_t>& rp, std::vector<int32_t>& col,
              std::vector<int64_t>& w) {
  std::vector<int64_t> off;
  std::vector<int32_t> len, pc;
  std::vector<WT> pw;
  dl(c, off, g.off.p, (size_t)rows);
  dl(c, len, g.len.p, (size_t)rows);
  dl(c, pc, g.col.p, (size_t)g.pool_top);
  dl(c, pw, g.w.p, (size_t)g.pool_top);
  CK(cudaStreamSynchronize(c.s));
  rp.assign((size_t)rows + 1, 0);
  for (int64_t v = 0; v < rows; ++v) rp[v + 1] = rp[v] + len[v];
  col.resize((size_t)rp[rows]);
  w.resize((size_t)rp[rows]);
  for (int64_t v = 0; v < rows; ++v)
    for (int32_t k = 0; k < len[v]; ++k) {
      col[rp[v] + k] = pc[off[v] + k];
      w[rp[v] + k] = (int64_t)pw[off[v] + k];
    }
}

void save_image(ldl_ctx& c, Image& im) {
  const size_t n = (size_t)c.n;
  im.prm = c.prm;
  im.prm.cuda_stream = nullptr;
  im.n = c.n;
  im.T = c.T;
  im.m = c.m;
  im.E = c.E;
  im.P_hi = (int64_t)(c.Psum >> 64);
  im.P_lo = (uint64_t)c.Psum;
  dl(c, im.Kout, c.Kout.p, n);
  if (c.directed) dl(c, im.Kin, c.Kin.p, n);
  dl(c, im.e, c.e.p, n);
  im.lv.assign((size_t)c.T + 1, LevelImage());
  const int64_t rows = c.directed ? 2 * c.n : c.n;
  for (int r = 0; r <= c.T; ++r) {
    LevelState& L = c.lv[r];
    LevelImage& I = im.lv[(size_t)r];
    dl(c, I.lab, L.lab.p, n);
    dl(c, I.par, L.par.p, n);
    dl(c, I.cnt, L.cnt.p, n);
    dl(c, I.kout, L.kout.p, n);
    if (c.directed) dl(c, I.kin, L.kin.p, n);
    dl(c, I.alive, L.alive.p, n);
    if (r == 0) csr_rows(c, L.out0, rows, I.rp, I.col, I.w);
    else csr_rows(c, L.out, rows, I.rp, I.col, I.w);
    if (r < c.T) {
      std::vector<int64_t> cw;
      csr_rows(c, L.children, c.n, I.crp, I.ccol, cw);
    }
    if (r == c.T) std::fill(I.par.begin(), I.par.end(), -1);
  }
  CK(cudaStreamSynchronize(c.s));
}

template <class T>
void ul(ldl_ctx& c, T* dst, const std::vector<T>& src) {
  if (!src.empty()) CK(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, c.s));
}

// Builds a slack CSR from compact sorted rows.
template <class WT>
void build_rows(ldl_ctx& c, SlackCSR<WT>& g, int64_t rows, const std::vector<int64_t>& rp,
                const std::vector<int32_t>& col, const std::vector<int64_t>* w) {
  const int64_t nrec = rp[(size_t)rows];
  std::vector<u64> keys((size_t)nrec);
  std::vector<int64_t> vals((size_t)nrec, 1);
  for (int64_t v = 0; v < rows; ++v)
    for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
      keys[(size_t)k] = ((u64)v << c.bits) | (u64)col[(size_t)k];
      if (w) vals[(size_t)k] = (*w)[(size_t)k];
    }
  c.rk.reserve(nrec + 1, c.s);
  c.rsum.reserve(nrec + 1, c.s);
  ul(c, c.rk.p, keys);
  ul(c, c.rsum.p, vals);
  csr_build<WT>(g, rows, c.rk.p, c.rsum.p, nrec, c.bits, 25, c.CS, c.P, c.s);
  CK(cudaStreamSynchronize(c.s));
}

void load_image(ldl_ctx& c, const Image& im) {
  const int64_t rows = c.directed ? 2 * c.n : c.n;
  c.T = im.T;
  c.m = im.m;
  c.E = im.E;
  c.Psum = i128_of(im.P_hi, im.P_lo);
  ul(c, c.Kout.p, im.Kout);
  if (c.directed) ul(c, c.Kin.p, im.Kin);
  ul(c, c.e.p, im.e);
  for (int r = 0; r <= im.T; ++r) {
    level_alloc(c, r);
    LevelState& L = c.lv[r];
    const LevelImage& I = im.lv[(size_t)r];
    ul(c, L.lab.p, I.lab);
    ul(c, L.par.p, I.par);
    ul(c, L.cnt.p, I.cnt);
    ul(c, L.kout.p, I.kout);
    if (c.directed) ul(c, L.kin.p, I.kin);
    ul(c, L.alive.p, I.alive);
    if (r == 0) build_rows<int32_t>(c, L.out0, rows, I.rp, I.col, &I.w);
    else build_rows<int64_t>(c, L.out, rows, I.rp, I.col, &I.w);
    if (r < im.T) build_rows<int32_t>(c, L.children, c.n, I.crp, I.ccol, nullptr);
  }
  CK(cudaStreamSynchronize(c.s));
}

// Appends isolated vertices n..n_new-1: each is its own community and, at
// every level, its own node (named by its id) whose parent is the node of the
// same id one level up, so the hierarchy's invariants hold; strengths and
// community totals are zero, so the modularity is unchanged.
void grow_image(Image& im, int64_t n_new) {
  const int64_t n = im.n;
  const bool directed = im.prm.directed != 0;
  auto ext = [&](auto& v, auto fill) { v.resize((size_t)n_new, fill); };
  ext(im.Kout, (int64_t)0);
  if (directed) ext(im.Kin, (int64_t)0);
  ext(im.e, (int64_t)0);
  for (int r = 0; r <= im.T; ++r) {
    LevelImage& I = im.lv[(size_t)r];
    I.lab.resize((size_t)n_new);
    I.par.resize((size_t)n_new);
    for (int64_t v = n; v < n_new; ++v) {
      I.lab[(size_t)v] = (int32_t)v;
      I.par[(size_t)v] = r < im.T ? (int32_t)v : -1;
    }
    ext(I.cnt, (int32_t)1);
    ext(I.kout, (int64_t)0);
    if (directed) ext(I.kin, (int64_t)0);
    ext(I.alive, (uint8_t)1);
    // adjacency rows: the new vertices' out-rows (empty) follow the old
    // out-rows; directed in-rows move behind them and gain empty rows too
    std::vector<int64_t> rp;
    std::vector<int32_t> col;
    std::vector<int64_t> w;
    const int64_t parts = directed ? 2 : 1;
    rp.push_back(0);
    for (int64_t p = 0; p < parts; ++p) {
      for (int64_t v = 0; v < n; ++v) {
        const int64_t row = p * n + v;
        for (int64_t k = I.rp[(size_t)row]; k < I.rp[(size_t)row + 1]; ++k) {
          col.push_back(I.col[(size_t)k]);
          w.push_back(I.w[(size_t)k]);
        }
        rp.push_back((int64_t)col.size());
      }
      for (int64_t v = n; v < n_new; ++v) rp.push_back((int64_t)col.size());
    }
    I.rp.swap(rp);
    I.col.swap(col);
    I.w.swap(w);
    if (r < im.T) {  // node v one level up has the single child v
      for (int64_t v = n; v < n_new; ++v) {
        I.ccol.push_back((int32_t)v);
        I.crp.push_back((int64_t)I.ccol.size());
      }
    }
  }
  im.n = n_new;
}

// ---- file format: a magic word, the parameters and sizes, then every array
// as (element count, bytes)
const char MAGIC[8] = {'L', 'D', 'L', 'H', 'I', 'E', 'R', '1'};

struct Writer {
  FILE* f;
  bool ok = true;
  void raw(const void* p, size_t b) { ok = ok && (b == 0 || fwrite(p, 1, b, f) == b); }
  template <class T>
  void val(const T& v) { raw(&v, sizeof(T)); }
  template <class T>
  void vec(const std::vector<T>& v) {
    val((int64_t)v.size());
    raw(v.data(), sizeof(T) * v.size());
  }
};

struct Reader {
  FILE* f;
  bool ok = true;
  void raw(void* p, size_t b) { ok = ok && (b == 0 || fread(p, 1, b, f) == b); }
  template <class T>
  void val(T& v) { raw(&v, sizeof(T)); }
  template <class T>
  void vec(std::vector<T>& v, int64_t limit) {
    int64_t k = -1;
    val(k);
    if (!ok || k < 0 || k > limit) {
      ok = false;
      return;
    }
    v.resize((size_t)k);
    raw(v.data(), sizeof(T) * v.size());
  }
};

bool write_image(const Image& im, const char* path) {
  FILE* f = fopen(path, "wb");
  if (!f) return false;
  Writer w{f};
  w.raw(MAGIC, sizeof MAGIC);
  ldl_params p = im.prm;
  p.cuda_stream = nullptr;
  w.val(p);
  w.val(im.n);
  w.val(im.T);
  w.val(im.m);
  w.val(im.E);
  w.val(im.P_hi);
  w.val(im.P_lo);
  w.vec(im.Kout);
  w.vec(im.Kin);
  w.vec(im.e);
  for (const LevelImage& I : im.lv) {
    w.vec(I.lab); w.vec(I.par); w.vec(I.cnt); w.vec(I.kout); w.vec(I.kin); w.vec(I.alive);
    w.vec(I.rp); w.vec(I.col); w.vec(I.w); w.vec(I.crp); w.vec(I.ccol);
  }
  const bool ok = w.ok;
  return fclose(f) == 0 && ok;
}

bool read_image(Image& im, const char* path, std::string& why) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    why = "cannot open the file";
    return false;
  }
  Reader r{f};
  char magic[8];
  r.raw(magic, sizeof magic);
  if (!r.ok || memcmp(magic, MAGIC, sizeof magic) != 0) {
    fclose(f);
    why = "not a hierarchy checkpoint";
    return false;
  }
  r.val(im.prm);
  im.prm.cuda_stream = nullptr;
  r.val(im.n);
  r.val(im.T);
  r.val(im.m);
  r.val(im.E);
  r.val(im.P_hi);
  r.val(im.P_lo);
  const int64_t n = im.n;
  if (!r.ok || n <= 0 || n > INT32_MAX - 1 || im.T < 0 || im.T > im.prm.L || im.prm.L > 7) {
    fclose(f);
    why = "corrupt header";
    return false;
  }
  const int64_t big = (int64_t)1 << 40;
  r.vec(im.Kout, n);
  r.vec(im.Kin, n);
  r.vec(im.e, n);
  im.lv.assign((size_t)im.T + 1, LevelImage());
  for (LevelImage& I : im.lv) {
    r.vec(I.lab, n); r.vec(I.par, n); r.vec(I.cnt, n); r.vec(I.kout, n); r.vec(I.kin, n); r.vec(I.alive, n);
    r.vec(I.rp, 2 * n + 1); r.vec(I.col, big); r.vec(I.w, big); r.vec(I.crp, n + 1); r.vec(I.ccol, n);
  }
  fclose(f);
  if (!r.ok) {
    why = "truncated or corrupt file";
    return false;
  }
  // structural checks: sizes, row tables, ids in range
  const bool directed = im.prm.directed != 0;
  const int64_t rows = directed ? 2 * n : n;
  auto bad = [&](const char* w2) {
    why = w2;
    return false;
  };
  if ((int64_t)im.Kout.size() != n || (int64_t)im.e.size() != n || (directed && (int64_t)im.Kin.size() != n))
    return bad("community totals of the wrong size");
  for (int t = 0; t <= im.T; ++t) {
    const LevelImage& I = im.lv[(size_t)t];
    if ((int64_t)I.lab.size() != n || (int64_t)I.par.size() != n || (int64_t)I.cnt.size() != n ||
        (int64_t)I.kout.size() != n || (int64_t)I.alive.size() != n || (directed && (int64_t)I.kin.size() != n))
      return bad("level arrays of the wrong size");
    if ((int64_t)I.rp.size() != rows + 1 || I.rp[0] != 0 || I.rp[(size_t)rows] != (int64_t)I.col.size() ||
        I.w.size() != I.col.size())
      return bad("adjacency row table inconsistent");
    for (int64_t v = 0; v < rows; ++v)
      if (I.rp[(size_t)v + 1] < I.rp[(size_t)v]) return bad("adjacency row table not monotone");
    for (size_t k = 0; k < I.col.size(); ++k)
      if (I.col[k] < 0 || I.col[k] >= n) return bad("adjacency id out of range");
    for (int64_t v = 0; v < n; ++v)
      if (I.lab[(size_t)v] < 0 || I.lab[(size_t)v] >= n || I.par[(size_t)v] < -1 || I.par[(size_t)v] >= n)
        return bad("label or parent out of range");
    if (t < im.T) {
      if ((int64_t)I.crp.size() != n + 1 || I.crp[0] != 0 || I.crp[(size_t)n] != (int64_t)I.ccol.size())
        return bad("children row table inconsistent");
      for (int64_t v = 0; v < n; ++v)
        if (I.crp[(size_t)v + 1] < I.crp[(size_t)v]) return bad("children row table not monotone");
      for (int32_t x : I.ccol)
        if (x < 0 || x >= n) return bad("child id out of range");
    }
  }
  return true;
}

}  // namespace

extern "C" {

ldl_status ldl_save(const ldl_ctx* cc, const char* path) {
  if (!cc || !path) return LDL_E_INVALID;
  ldl_ctx& c = const_cast<ldl_ctx&>(*cc);
  try {
    DeviceScope ds(c.dev);
    Image im;
    save_image(c, im);
    if (!write_image(im, path)) {
      c.err = std::string("ldl_save: cannot write ") + path;
      return LDL_E_INVALID;
    }
  } catch (const LdlError& e) {
    c.err = e.msg;
    cudaGetLastError();
    return e.st;
  }
  return LDL_OK;
}

ldl_status ldl_load(const char* path, const ldl_params* params, ldl_ctx** out) {
  if (!path || !out) return LDL_E_INVALID;
  *out = nullptr;
  Image im;
  std::string why;
  if (!read_image(im, path, why)) {
    set_create_error(std::string("ldl_load: ") + why);
    return LDL_E_INVALID;
  }
  ldl_params p = im.prm;
  if (params) {  // the caller's stream and scheduling knobs; the method's parameters stay as saved
    p.cuda_stream = params->cuda_stream;
    p.kernel_stats = params->kernel_stats;
    p.cluster_max_deg = params->cluster_max_deg;
    p.no_rollback = params->no_rollback;
    for (int i = 0; i < 4; ++i) p.bin_deg[i] = params->bin_deg[i];
  }
  ldl_ctx* c = nullptr;
  const ldl_status st = ctx_new(p, im.n, &c);
  if (st != LDL_OK) return st;
  try {
    load_image(*c, im);
  } catch (const LdlError& e) {
    set_create_error(e.msg);
    free_all(*c);
    delete c;
    cudaGetLastError();
    return e.st;
  }
  *out = c;
  return LDL_OK;
}

ldl_status ldl_grow(ldl_ctx* c, int64_t n_new) {
  if (!c) return LDL_E_INVALID;
  if (n_new < c->n || n_new > INT32_MAX - 1) {
    c->err = "ldl_grow: the new vertex count must be at least n and at most 2^31-2";
    return LDL_E_INVALID;
  }
  if (n_new == c->n) return LDL_OK;
  if (c->broken) {
    c->err = "the context's state was lost by an earlier failed rollback; destroy it";
    return LDL_E_CUDA;
  }
  try {
    DeviceScope ds(c->dev);
    Image im;
    save_image(*c, im);
    grow_image(im, n_new);
    // a context of the new size is set up beside the old one, so that a
    // failure leaves the old state untouched; then the two swap contents
    ldl_params p = c->prm;
    ldl_ctx* fresh = nullptr;
    const ldl_status st = ctx_new(p, n_new, &fresh);
    if (st != LDL_OK) {
      c->err = "ldl_grow: cannot set up the larger context";
      return st;
    }
    try {
      load_image(*fresh, im);
    } catch (...) {
      free_all(*fresh);
      delete fresh;
      throw;
    }
    fresh->epoch = c->epoch;
    std::swap(*c, *fresh);
    c->P.rd_owner = c;  // the scan primitives read counters back through their context
    fresh->P.rd_owner = fresh;
    free_all(*fresh);
    delete fresh;
  } catch (const LdlError& e) {
    c->err = e.msg;
    cudaGetLastError();
    return e.st;
  }
  return LDL_OK;
}

}  // extern "C"
