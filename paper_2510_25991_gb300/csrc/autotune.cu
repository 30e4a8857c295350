// autotune.cu -- the autotuner and its cache file (host code).
//
// The method fixes what is computed (Alg. 1, Alg. 2, the GMRES solve of Sec. 1, Eq. (modelS)),
// not the schedule: how each pivot sweep is split into warm-started chunks, the tensor-core
// precision of the local operators, whether the transfer operators are formed (Alg. 1) or
// applied through local solves (Sec. 2.5), and how the inner GMRES tolerance is balanced against
// FP64 refinement steps.  The tuner times these knobs on the caller's own problems through the
// public entry points, one knob at a time starting from the automatic choices, and keeps a
// candidate only if the refinement still contracts by at least a factor 10 per step: a faster
// but less accurate operator must not buy its speed with a refinement that barely converges.
// The result is cached in a text file under a key made of the device and the problem shapes;
// ddst_setup applies a cached entry to the knobs the caller left automatic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include <unistd.h>

#include "../../include/ddst.h"

namespace ddst {
void set_global_error(const std::string& m);  // message for ddst_last_error(NULL), api.cu
}

namespace {

constexpr double kTuneRhoMax = 0.1;   // slowest refinement contraction a candidate may show
constexpr double kTuneMinGain = 0.02; // a candidate replaces the best only if 2% faster

ddst_status arg_error(const char* m) {
  ddst::set_global_error(m);
  return DDST_ERR_INVALID_ARG;
}

std::string make_key(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                     const int* widths, int precision) {
  std::string dev = "nodevice";
  int d = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&d) == cudaSuccess && cudaGetDeviceProperties(&p, d) == cudaSuccess) {
    std::string name = p.name;
    for (char& c : name)
      if (c == ' ' || c == '\t' || c == ';' || c == ',') c = '_';
    dev = name + "/sm" + std::to_string(p.major) + std::to_string(p.minor) + "/" +
          std::to_string(p.multiProcessorCount);
  } else {
    cudaGetLastError();  // no device here: the key says so
  }
  std::string key = "dev=" + dev + ";prec=" + std::to_string(precision) + ";probs=";
  for (int q = 0; q < nprob; ++q) {
    if (q) key += ",";
    key += "d" + std::to_string(grids[q].dim) + "n" + std::to_string((long long)grids[q].n) +
           "w" + std::to_string(widths[q]) + (coeffs[q].c ? "c" : "");
  }
  return key;
}

std::string format_knobs(const ddst_options& o) {
  char buf[256];
  snprintf(buf, sizeof(buf),
           "precision=%d tensor_cores=%d explicit_S=%d gmres_tol=%.17g check_every=%d "
           "factor_chunks=%d interface_solver=%d",
           o.precision, o.tensor_cores, o.explicit_S, o.gmres_tol, o.check_every,
           o.factor_chunks, o.interface_solver);
  return buf;
}

struct Knobs {
  int precision = DDST_MIXED, tensor_cores = 1, explicit_S = -1, check_every = 0,
      factor_chunks = 0, interface_solver = 0;
  double gmres_tol = 0.0;
};

// Parses "name=value" tokens; false if a knob is missing or malformed.
bool parse_knobs(const std::string& s, Knobs* k) {
  std::istringstream in(s);
  std::string tok;
  int seen = 0;
  while (in >> tok) {
    const size_t eq = tok.find('=');
    if (eq == std::string::npos) return false;
    const std::string name = tok.substr(0, eq), val = tok.substr(eq + 1);
    char* end = nullptr;
    if (name == "gmres_tol") {
      k->gmres_tol = strtod(val.c_str(), &end);
    } else {
      const long v = strtol(val.c_str(), &end, 10);
      if (name == "precision") k->precision = (int)v;
      else if (name == "tensor_cores") k->tensor_cores = (int)v;
      else if (name == "explicit_S") k->explicit_S = (int)v;
      else if (name == "check_every") k->check_every = (int)v;
      else if (name == "factor_chunks") k->factor_chunks = (int)v;
      else if (name == "interface_solver") k->interface_solver = (int)v;
      else continue;  // a knob of a later version: ignored
    }
    if (!end || *end != '\0') return false;
    ++seen;
  }
  return seen == 7 && (k->precision == DDST_FP64 || k->precision == DDST_MIXED ||
                       k->precision == DDST_MIXED_TF32);
}

// The knobs the caller left automatic take the tuned values.
void apply_knobs(const Knobs& k, ddst_options* o) {
  if (o->precision == DDST_AUTO) o->precision = k.precision;
  if (o->tensor_cores < 0) o->tensor_cores = k.tensor_cores;
  if (o->explicit_S < 0) o->explicit_S = k.explicit_S;
  if (!(o->gmres_tol > 0.0)) o->gmres_tol = k.gmres_tol;
  if (o->check_every == 0) o->check_every = k.check_every;
  if (o->factor_chunks == 0) o->factor_chunks = k.factor_chunks;
  if (o->interface_solver < 0) o->interface_solver = k.interface_solver;
}

bool read_lines(const char* path, std::vector<std::string>* lines) {
  std::ifstream in(path);
  if (!in) return false;
  std::string line;
  while (std::getline(in, line)) lines->push_back(line);
  return true;
}

struct Eval {
  ddst_status st = DDST_OK;
  double ms = 0.0, rho = 0.0;
  int chunks = 0;
  bool matfree_only = false;
};

// One candidate: setup, transfer build, compression, two solves.  Cost in event milliseconds:
// the setup phases, the direct interface factorization (once), and `solves` times the second
// solve (the first also pays one-time work: graph capture, the direct factorization).
Eval evaluate(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs, const int* widths,
              const double* const* f, const double* const* g, double* const* u,
              double compress_tol, int solves, const ddst_options& o, void* stream) {
  Eval r;
  ddst_ctx* ctx = nullptr;
  r.st = ddst_setup_batch(nprob, grids, coeffs, widths, &o, stream, &ctx);
  if (r.st != DDST_OK) return r;
  ddst_info i1, i2;
  r.st = ddst_build_transfer(ctx);
  if (r.st == DDST_OK && compress_tol > 0.0) r.st = ddst_compress(ctx, compress_tol);
  if (r.st == DDST_OK) r.st = ddst_solve_batch(ctx, f, g, u, &i1);
  if (r.st == DDST_OK) r.st = ddst_solve_batch(ctx, f, g, u, &i2);
  if (r.st == DDST_OK) {
    r.ms = i2.t_factor + i2.t_transfer + i2.t_compress + i2.t_direct + solves * i2.t_solve;
    r.rho = std::max(i1.refine_rho, i2.refine_rho);
    r.chunks = i2.factor_chunks;
  }
  ddst_destroy(ctx);
  return r;
}

}  // namespace

extern "C" {

ddst_status ddst_partition(int nitems, const double* cost, int world, int* owner,
                           double* load) {
  if (nitems < 0 || world <= 0 || (nitems > 0 && (!cost || !owner)))
    return arg_error("ddst_partition: bad sizes or NULL argument");
  for (int i = 0; i < nitems; ++i)
    if (!(cost[i] >= 0.0)) return arg_error("ddst_partition: costs must be >= 0");
  // longest processing time first: items by decreasing cost (ties by index), each to the rank
  // with the least load so far (ties by rank)
  std::vector<int> order(nitems);
  for (int i = 0; i < nitems; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> ld(world, 0.0);
  for (int i : order) {
    int r = 0;
    for (int k = 1; k < world; ++k)
      if (ld[k] < ld[r]) r = k;
    owner[i] = r;
    ld[r] += cost[i];
  }
  if (load)
    for (int k = 0; k < world; ++k) load[k] = ld[k];
  return DDST_OK;
}

ddst_status ddst_autotune_key(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                              const int* slab_widths, int precision, char* buf, size_t len) {
  if (nprob <= 0 || !grids || !coeffs || !slab_widths || !buf)
    return arg_error("ddst_autotune_key: bad problem list or NULL buffer");
  const std::string key = make_key(nprob, grids, coeffs, slab_widths, precision);
  if (key.size() + 1 > len) return arg_error("ddst_autotune_key: buffer too small");
  memcpy(buf, key.c_str(), key.size() + 1);
  return DDST_OK;
}

ddst_status ddst_autotune_lookup(const char* path, const char* key, ddst_options* opt,
                                 int* found) {
  if (!path || !key || !opt || !found) return arg_error("ddst_autotune_lookup: NULL argument");
  *found = 0;
  std::vector<std::string> lines;
  if (!read_lines(path, &lines)) return DDST_OK;  // no cache yet
  const std::string k = key;
  for (const std::string& line : lines) {
    const size_t tab = line.find('\t');
    if (tab == std::string::npos || line.compare(0, tab, k) != 0 || tab != k.size()) continue;
    Knobs kn;
    if (!parse_knobs(line.substr(tab + 1), &kn)) continue;
    apply_knobs(kn, opt);
    *found = 1;  // the last valid entry wins (the store keeps one per key)
  }
  return DDST_OK;
}

ddst_status ddst_autotune_store(const char* path, const char* key, const ddst_options* opt) {
  if (!path || !key || !opt) return arg_error("ddst_autotune_store: NULL argument");
  if (strchr(key, '\t') || strchr(key, '\n')) return arg_error("ddst_autotune_store: bad key");
  std::vector<std::string> lines, keep;
  read_lines(path, &lines);
  const std::string k = key;
  for (const std::string& line : lines) {
    const size_t tab = line.find('\t');
    if (tab != std::string::npos && tab == k.size() && line.compare(0, tab, k) == 0) continue;
    if (!line.empty()) keep.push_back(line);
  }
  keep.push_back(k + "\t" + format_knobs(*opt));
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
  {
    std::ofstream out(tmp, std::ios::trunc);
    if (!out) return arg_error("ddst_autotune_store: cannot write the cache file");
    for (const std::string& line : keep) out << line << "\n";
    if (!out.good()) return arg_error("ddst_autotune_store: cannot write the cache file");
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return arg_error("ddst_autotune_store: cannot replace the cache file");
  }
  return DDST_OK;
}

ddst_status ddst_autotune(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                          const int* slab_widths, const double* const* f,
                          const double* const* g, double compress_tol, int solves_per_setup,
                          const ddst_options* base, void* stream, ddst_tune_report* rep) {
  if (nprob <= 0 || !grids || !coeffs || !slab_widths || !f || !g || !rep)
    return arg_error("ddst_autotune: bad problem list or NULL argument");
  const int solves = std::max(1, solves_per_setup);
  for (int q = 0; q < nprob; ++q)
    if (!f[q] || !g[q]) return arg_error("ddst_autotune: NULL right-hand side");
  ddst_options b;
  if (base) b = *base; else ddst_options_default(&b);
  memset(rep, 0, sizeof(*rep));
  const char* cache = b.autotune_cache;
  b.autotune_cache = nullptr;  // candidates run exactly as given
  // output buffers on the device
  std::vector<double*> u(nprob, nullptr);
  auto free_u = [&]() {
    for (double* p : u) cudaFree(p);
  };
  for (int q = 0; q < nprob; ++q) {
    size_t n = 1;
    for (int d = 0; d < grids[q].dim; ++d) n *= (size_t)std::max<int64_t>(grids[q].n - 1, 1);
    if (cudaMalloc(&u[q], sizeof(double) * n) != cudaSuccess) {
      cudaGetLastError();
      free_u();
      ddst::set_global_error("ddst_autotune: cudaMalloc of the solution buffers failed");
      return DDST_ERR_OOM;
    }
  }
  const int req_prec = b.precision;
  ddst_options cur = b;
  if (cur.precision == DDST_AUTO) cur.precision = DDST_MIXED;
  if (cur.tensor_cores < 0) cur.tensor_cores = 1;
  if (cur.interface_solver < 0) cur.interface_solver = 0;
  auto run = [&](const ddst_options& o) {
    ++rep->candidates;
    Eval e = evaluate(nprob, grids, coeffs, slab_widths, f, g, u.data(), compress_tol, solves, o,
                      stream);
    if (e.st != DDST_OK || !(e.rho <= kTuneRhoMax)) ++rep->rejected;
    return e;
  };
  // the untuned configuration, twice: the first run also pays one-time module loading
  run(cur);
  Eval best = run(cur);
  if (best.st == DDST_ERR_SINGULAR && req_prec == DDST_AUTO) {  // DDST_AUTO's FP64 fallback
    cur.precision = DDST_FP64;
    best = run(cur);
  }
  if (best.st != DDST_OK) {
    free_u();
    return best.st;
  }
  rep->default_ms = best.ms;
  auto consider = [&](ddst_options cand) {
    const Eval e = run(cand);
    if (e.st == DDST_OK && e.rho <= kTuneRhoMax && e.ms < (1.0 - kTuneMinGain) * best.ms) {
      best = e;
      cur = cand;
    }
  };
  const bool mixed = cur.precision != DDST_FP64;
  // 1. explicit S or matrix-free (compression needs the explicit operators)
  if (b.explicit_S < 0 && !(compress_tol > 0.0)) {
    ddst_options c = cur;
    c.explicit_S = 0;
    consider(c);
  }
  // 2. interface solver: GMRES or the block cyclic reduction (explicit operators only)
  if (b.interface_solver < 0 && cur.explicit_S != 0) {
    ddst_options c = cur;
    c.interface_solver = 1;
    consider(c);
  }
  // 3. tensor-core precision of the local operators
  if (mixed) {
    if (b.tensor_cores < 0) {
      ddst_options c = cur;
      c.tensor_cores = 0;
      c.precision = DDST_MIXED;
      consider(c);
    }
    if (req_prec == DDST_AUTO) {
      ddst_options c = cur;
      c.precision = DDST_MIXED_TF32;
      c.tensor_cores = 1;
      consider(c);
    }
  }
  // 4. inner GMRES tolerance against refinement steps
  if (!(b.gmres_tol > 0.0) && cur.interface_solver != 1) {
    const std::vector<double> tols = mixed ? std::vector<double>{1e-2, 1e-3, 1e-4}
                                           : std::vector<double>{1e-8, 1e-10};
    for (double t : tols) {
      ddst_options c = cur;
      c.gmres_tol = t;
      consider(c);
    }
  }
  // 5. host convergence checks of GMRES
  if (b.check_every == 0 && cur.interface_solver != 1)
    for (int ce : {1, 4, 16}) {
      ddst_options c = cur;
      c.check_every = ce;
      consider(c);
    }
  // 6. warm-started chunks of the pivot sweeps (around the automatic count)
  if (b.factor_chunks == 0 && best.chunks > 1) {
    const int used = best.chunks;
    for (int k : {1, std::max(2, used / 2), used * 2}) {
      if (k == used) continue;
      ddst_options c = cur;
      c.factor_chunks = k;
      consider(c);
    }
  }
  free_u();
  rep->best_ms = best.ms;
  rep->best_rho = best.rho;
  rep->chosen = cur;
  rep->chosen.autotune_cache = cache;
  if (cache) {
    const std::string key = make_key(nprob, grids, coeffs, slab_widths, req_prec);
    const ddst_status s = ddst_autotune_store(cache, key.c_str(), &cur);
    if (s != DDST_OK) return s;
    rep->cache_written = 1;
  }
  return DDST_OK;
}

}  // extern "C"
