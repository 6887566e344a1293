// extern "C" entry points of libctq (declared in include/ctq.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctq_internal.h"

struct ctq_impurity {
  ctq::HostModel host;
  int device = -1;
  int num_sms = 0;
  ctq::DevModel dev{};
  ctq::LaunchCfg launch{};
  const int64_t* rho_off = nullptr;  // density-matrix sector offsets (device)
  int optin = 0;                     // opt-in shared memory per block
  // tensor-core path (real impurities with blocks <= 112): TF32 and 3xTF32
  ctq::TcParams tc1{}, tc2{}, tc3{};  // CTQ_TF32, CTQ_BF16X3, CTQ_TF32X3
  ctq::LaunchCfg launch_tc1{}, launch_tc2{}, launch_tc3{};
  // large-block tensor-core path (complex impurities or blocks > 112)
  bool big = false;
  bool big64 = false;  // CTQ_FP64 on the float64 large-block kernel
  ctq::Big64Params b64{};
  ctq::LaunchCfg launch_b64{};
  ctq::BigParams big1{}, big2{}, big3{};  // CTQ_TF32, CTQ_BF16X3, CTQ_TF32X3
  ctq::LaunchCfg launch_big1{}, launch_big2{}, launch_big3{};
  std::vector<void*> allocs;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    ok_ = (dev == prev_) || cudaSetDevice(dev) == cudaSuccess;
    switched_ = dev != prev_;
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }

 private:
  int prev_ = 0;
  bool ok_ = false, switched_ = false;
};

template <typename T>
int upload_vec(ctq_impurity* imp, const std::vector<T>& v, const T** dst) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
  if (cudaMalloc(&p, bytes) != cudaSuccess) return CTQ_ERR_NOMEM;
  imp->allocs.push_back(p);
  if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return CTQ_ERR_CUDA;
  *dst = static_cast<const T*>(p);
  return CTQ_OK;
}

void free_device(ctq_impurity* imp) {
  if (imp->device < 0) return;
  DeviceGuard g(imp->device);
  for (void* p : imp->allocs) cudaFree(p);
  imp->allocs.clear();
}

// Copies the host model to its device: energies relative to each sector's
// minimum, sector map, block offsets, blocks (complex interleaved) and
// log spectral norms.
int upload_model(ctq_impurity* imp) {
  const ctq::HostModel& h = imp->host;
  if (imp->device < 0) return CTQ_OK;
  DeviceGuard g(imp->device);
  if (!g.ok()) return fail(CTQ_ERR_CUDA, "cudaSetDevice failed");
  if (cudaDeviceGetAttribute(&imp->num_sms, cudaDevAttrMultiProcessorCount, imp->device) != cudaSuccess)
    return fail(CTQ_ERR_CUDA, "cannot query the device");
  ctq::DevModel& d = imp->dev;
  d.n_flav = h.n_flav;
  d.n_alpha = h.n_alpha();
  d.n_sec = h.n_sec;
  d.max_dim = h.max_dim;
  d.is_complex = h.is_complex;
  d.E_ref = h.E_gs;
  std::vector<double> e_rel(h.E.size());
  for (int q = 0; q < h.n_sec; ++q)
    for (int j = h.E_off[q]; j < h.E_off[q + 1]; ++j) e_rel[j] = h.E[j] - h.E_min[q];
  std::vector<float> e_relf(e_rel.begin(), e_rel.end());
  std::vector<double> lev_E;
  std::vector<int> lev_off(1, 0), lev_idx(h.E.size());
  for (int q = 0; q < h.n_sec; ++q) {
    const int base = int(lev_E.size());
    for (int j = h.E_off[q]; j < h.E_off[q + 1]; ++j) {
      int l = base;
      while (l < int(lev_E.size()) && lev_E[l] != e_rel[j]) ++l;  // bitwise equal values only
      if (l == int(lev_E.size())) lev_E.push_back(e_rel[j]);
      lev_idx[j] = l - base;
    }
    lev_off.push_back(int(lev_E.size()));
  }
  d.max_lev = 1;
  for (int q = 0; q < h.n_sec; ++q) d.max_lev = std::max(d.max_lev, lev_off[q + 1] - lev_off[q]);
  std::vector<double> blk;
  if (h.is_complex) {
    blk.resize(2 * h.blk_re.size());
    for (size_t i = 0; i < h.blk_re.size(); ++i) {
      blk[2 * i] = h.blk_re[i];
      blk[2 * i + 1] = h.blk_im[i];
    }
  } else {
    blk = h.blk_re;
  }
  std::vector<double> log_dim(h.dims.size());
  for (size_t q = 0; q < log_dim.size(); ++q) log_dim[q] = std::log(double(h.dims[q]));
  std::vector<double> lognorm(h.opnorm.size());
  for (size_t i = 0; i < lognorm.size(); ++i) lognorm[i] = h.opnorm[i] > 0 ? std::log(h.opnorm[i]) : -INFINITY;
  int st = CTQ_OK;
  if ((st = upload_vec(imp, h.dims, &d.dims)) || (st = upload_vec(imp, log_dim, &d.log_dim)) ||
      (st = upload_vec(imp, h.E_off, &d.E_off)) ||
      (st = upload_vec(imp, e_rel, &d.E_rel)) || (st = upload_vec(imp, e_relf, &d.E_relf)) ||
      (st = upload_vec(imp, h.E_min, &d.E_min)) ||
      (st = upload_vec(imp, h.s, &d.s)) || (st = upload_vec(imp, h.blk_off, &d.blk_off)) ||
      (st = upload_vec(imp, blk, &d.blk)) || (st = upload_vec(imp, lognorm, &d.log_norm)) ||
      (st = upload_vec(imp, lev_E, &d.lev_E)) || (st = upload_vec(imp, lev_off, &d.lev_off)) ||
      (st = upload_vec(imp, lev_idx, &d.lev_idx))) {
    free_device(imp);
    return fail(st, "device upload failed");
  }
  {
    std::vector<int64_t> roff(h.n_sec);
    int64_t acc = 0;
    for (int q = 0; q < h.n_sec; ++q) {
      roff[q] = acc;
      acc += int64_t(h.dims[q]) * h.dims[q];
    }
    st = upload_vec(imp, roff, &imp->rho_off);
  }
  if (st == CTQ_OK &&
      cudaDeviceGetAttribute(&imp->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, imp->device) != cudaSuccess)
    st = CTQ_ERR_CUDA;
  if (st == CTQ_OK) st = ctq::prepare_rho(imp->optin);
  if (st != CTQ_OK) {
    free_device(imp);
    return fail(st, "device upload failed");
  }
  if ((st = ctq::prepare_eval_fp64(d, imp->num_sms, &imp->launch)) != CTQ_OK) {
    free_device(imp);
    return fail(st, "cannot configure the trace kernel");
  }
  if (ctq::fp64_shared_kernel_fits(d, imp->optin)) {
    // two-float copy of the blocks for CTQ_F32X2: hi = fl(x), lo = fl(x - hi)
    std::vector<float> bx(2 * blk.size());
    for (size_t i = 0; i < blk.size(); ++i) {
      const float hi = float(blk[i]);
      bx[2 * i] = hi;
      bx[2 * i + 1] = float(blk[i] - double(hi));
    }
    if ((st = upload_vec(imp, bx, &d.blk_x2)) != CTQ_OK) {
      free_device(imp);
      return fail(st, "device upload failed");
    }
  }
  if (!h.is_complex && h.max_dim <= 112) {
    std::vector<unsigned char> tcb, tcb16;
    std::vector<int64_t> tco, tco16;
    int stage3 = 0, stage2 = 0;
    const unsigned char *b3 = nullptr, *b2 = nullptr;
    if ((st = ctq::build_tc_blocks(h, CTQ_TF32X3, tcb, tco, &stage3)) != CTQ_OK ||
        (st = ctq::build_tc_blocks(h, CTQ_BF16X3, tcb16, tco16, &stage2)) != CTQ_OK ||
        (st = upload_vec(imp, tcb, &b3)) != CTQ_OK || (st = upload_vec(imp, tco, &imp->tc3.off)) != CTQ_OK ||
        (st = upload_vec(imp, tcb16, &b2)) != CTQ_OK || (st = upload_vec(imp, tco16, &imp->tc2.off)) != CTQ_OK) {
      free_device(imp);
      return fail(st, "tensor-core block upload failed");
    }
    imp->tc3.blk = b3;
    imp->tc2.blk = b2;
    imp->tc3.prec = CTQ_TF32X3;
    imp->tc3.stage_bytes = stage3;
    imp->tc3.tmem_cols = 512;
    imp->tc1 = imp->tc3;  // same blocks; TF32 fetches only the hi plane
    imp->tc1.prec = CTQ_TF32;
    imp->tc1.stage_bytes = stage3 / 2;
    imp->tc1.tmem_cols = 256;
    imp->tc2.prec = CTQ_BF16X3;
    imp->tc2.stage_bytes = stage2;
    imp->tc2.tmem_cols = 256;
    if ((st = ctq::prepare_eval_tc(d, CTQ_TF32X3, imp->tc3.stage_bytes, imp->num_sms, &imp->launch_tc3)) != CTQ_OK ||
        (st = ctq::prepare_eval_tc(d, CTQ_TF32, imp->tc1.stage_bytes, imp->num_sms, &imp->launch_tc1)) != CTQ_OK ||
        (st = ctq::prepare_eval_tc(d, CTQ_BF16X3, imp->tc2.stage_bytes, imp->num_sms, &imp->launch_tc2)) != CTQ_OK) {
      free_device(imp);
      return fail(st, "cannot configure the tensor-core kernel");
    }
  } else if (h.max_dim <= 3072) {
    // large blocks: embedded, tiled, split copies formatted on the device,
    // tf32 hi / lo (CTQ_TF32X3; CTQ_TF32 reads the hi planes) and bf16 hi / lo
    std::vector<int64_t> off(h.s.size(), -1);
    size_t total = 0;
    for (int a = 0; a < h.n_alpha(); ++a)
      for (int q = 0; q < h.n_sec; ++q) {
        const size_t i = size_t(a) * h.n_sec + q;
        if (h.s[i] < 0) continue;
        off[i] = int64_t(total);
        total += ctq::big_block_elems(h.dims[h.s[i]], h.dims[q]);
      }
    void *bt = nullptr, *bt16 = nullptr;
    if (cudaMalloc(&bt, std::max<size_t>(total, 1) * sizeof(float)) != cudaSuccess) {
      free_device(imp);
      return fail(CTQ_ERR_NOMEM, "cannot allocate the large-block operands");
    }
    imp->allocs.push_back(bt);
    if (cudaMalloc(&bt16, std::max<size_t>(total, 1) * sizeof(uint16_t)) != cudaSuccess) {
      free_device(imp);
      return fail(CTQ_ERR_NOMEM, "cannot allocate the large-block operands");
    }
    imp->allocs.push_back(bt16);
    if ((st = ctq::format_big_blocks(h, d.blk, bt, off, CTQ_TF32X3)) != CTQ_OK ||
        (st = ctq::format_big_blocks(h, d.blk, bt16, off, CTQ_BF16X3)) != CTQ_OK ||
        (st = upload_vec(imp, off, &imp->big3.bt_off)) != CTQ_OK) {
      free_device(imp);
      return fail(st, "large-block formatting failed");
    }
    imp->big3.bt = bt;
    imp->big3.prec = CTQ_TF32X3;
    imp->big1 = imp->big3;
    imp->big1.prec = CTQ_TF32;
    imp->big2 = imp->big3;
    imp->big2.bt = bt16;
    imp->big2.prec = CTQ_BF16X3;
    if ((st = ctq::prepare_eval_big(CTQ_TF32X3, imp->num_sms, &imp->launch_big3)) != CTQ_OK ||
        (st = ctq::prepare_eval_big(CTQ_TF32, imp->num_sms, &imp->launch_big1)) != CTQ_OK ||
        (st = ctq::prepare_eval_big(CTQ_BF16X3, imp->num_sms, &imp->launch_big2)) != CTQ_OK) {
      free_device(imp);
      return fail(st, "cannot configure the large-block kernel");
    }
    imp->big = true;
  }
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, imp->device) != cudaSuccess) {
    free_device(imp);
    return fail(CTQ_ERR_CUDA, "cannot query the device");
  }
  if (!ctq::fp64_shared_kernel_fits(d, optin) && h.max_dim <= 3072) {
    // float64 large-block path: embedded, row-major float64 copies of the blocks
    std::vector<int64_t> off(h.s.size(), -1);
    size_t total = 0;
    for (int a = 0; a < h.n_alpha(); ++a)
      for (int q = 0; q < h.n_sec; ++q) {
        const size_t i = size_t(a) * h.n_sec + q;
        if (h.s[i] < 0) continue;
        off[i] = int64_t(total);
        total += ctq::big64_block_elems(h.dims[h.s[i]], h.dims[q]);
      }
    // and the same as two-float pairs (CTQ_F32X2), 8 bytes per element too
    void* bt = nullptr;
    void* bx = nullptr;
    if (cudaMalloc(&bt, std::max<size_t>(total, 1) * sizeof(double)) != cudaSuccess) {
      free_device(imp);
      return fail(CTQ_ERR_NOMEM, "cannot allocate the float64 large-block operands");
    }
    imp->allocs.push_back(bt);
    if (cudaMalloc(&bx, std::max<size_t>(total, 1) * 2 * sizeof(float)) != cudaSuccess) {
      free_device(imp);
      return fail(CTQ_ERR_NOMEM, "cannot allocate the two-float large-block operands");
    }
    imp->allocs.push_back(bx);
    if ((st = ctq::format_big64_blocks(h, d.blk, bt, off, false)) != CTQ_OK ||
        (st = ctq::format_big64_blocks(h, d.blk, bx, off, true)) != CTQ_OK ||
        (st = upload_vec(imp, off, &imp->b64.bt_off)) != CTQ_OK ||
        (st = ctq::prepare_eval_big64(imp->num_sms, &imp->launch_b64)) != CTQ_OK) {
      free_device(imp);
      return fail(st, "float64 large-block setup failed");
    }
    imp->b64.bt = static_cast<const double*>(bt);
    imp->b64.bt_x2 = static_cast<const float*>(bx);
    imp->big64 = true;
  }
  return CTQ_OK;
}

// Power iteration on F^H F for ||F||_2 (user-supplied blocks).
double spectral_norm(int rows, int cols, const double* re, const double* im) {
  std::vector<double> xr(cols, 1.0 / std::sqrt(double(cols))), xi(cols, 0.0), yr(rows), yi(rows);
  double lam = 0.0;
  for (int it = 0; it < 200; ++it) {
    for (int r = 0; r < rows; ++r) {
      double ar = 0, ai = 0;
      for (int c = 0; c < cols; ++c) {
        const double fr = re[size_t(r) * cols + c], fi = im ? im[size_t(r) * cols + c] : 0.0;
        ar += fr * xr[c] - fi * xi[c];
        ai += fr * xi[c] + fi * xr[c];
      }
      yr[r] = ar;
      yi[r] = ai;
    }
    double nrm = 0;
    for (int c = 0; c < cols; ++c) {
      double ar = 0, ai = 0;
      for (int r = 0; r < rows; ++r) {
        const double fr = re[size_t(r) * cols + c], fi = im ? -im[size_t(r) * cols + c] : 0.0;
        ar += fr * yr[r] - fi * yi[r];
        ai += fr * yi[r] + fi * yr[r];
      }
      xr[c] = ar;
      xi[c] = ai;
      nrm += ar * ar + ai * ai;
    }
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) return 0.0;
    const double prev = lam;
    lam = nrm;
    for (int c = 0; c < cols; ++c) {
      xr[c] /= nrm;
      xi[c] /= nrm;
    }
    if (it > 5 && std::fabs(lam - prev) <= 1e-15 * lam) break;
  }
  return std::sqrt(lam) * (1.0 + 1e-9);
}

}  // namespace

namespace ctq {
void set_last_error(const std::string& msg) { g_last_error = msg; }
int impurity_device(const ctq_impurity* imp, int* device) {
  if (!imp || !device) return CTQ_ERR_ARG;
  *device = imp->device;
  return CTQ_OK;
}
const HostModel* impurity_host(const ctq_impurity* imp) { return imp ? &imp->host : nullptr; }
const DevModel* impurity_dev(const ctq_impurity* imp) { return imp ? &imp->dev : nullptr; }
void record_timing_event(void* event, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev = static_cast<cudaEvent_t>(event);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else
    cudaEventRecord(ev, st);
}
}  // namespace ctq

extern "C" {

const char* ctq_strerror(int code) {
  switch (code) {
    case CTQ_OK: return "ok";
    case CTQ_ERR_ARG: return "invalid argument";
    case CTQ_ERR_NOMEM: return "out of memory";
    case CTQ_ERR_CUDA: return "CUDA runtime error";
    case CTQ_ERR_TIMEOUT: return "device wait timed out";
    case CTQ_ERR_UNSUPPORTED: return "unsupported configuration";
    case CTQ_ERR_NUMERIC: return "eigensolver did not converge";
    case CTQ_ERR_WORKSPACE: return "workspace too small";
    default: return "unknown error";
  }
}

const char* ctq_last_error_message(void) { return g_last_error.c_str(); }

int ctq_build_impurity(const ctq_model_params* p, ctq_impurity** out) {
  if (!p || !out) return fail(CTQ_ERR_ARG, "null argument");
  *out = nullptr;
  try {
    ctq_impurity* imp = new ctq_impurity();
    std::string err;
    int st = ctq::build_host_model(p, imp->host, err);
    if (st != CTQ_OK) {
      delete imp;
      return fail(st, err);
    }
    imp->device = p->device;
    st = upload_model(imp);
    if (st != CTQ_OK) {
      delete imp;
      return st;
    }
    *out = imp;
    return CTQ_OK;
  } catch (const std::bad_alloc&) {
    return fail(CTQ_ERR_NOMEM, "host allocation failed");
  } catch (...) {
    return fail(CTQ_ERR_ARG, "unexpected exception");
  }
}

int ctq_load_impurity(int n_flav, int n_sec, const int* dims, const int* N, const double* energies,
                      const int* s_table, const double* blocks_re, const double* blocks_im,
                      const double* opnorm, double mu, int device, ctq_impurity** out) {
  if (!out || !dims || !energies || !s_table || !blocks_re || n_flav < 1 || n_sec < 1)
    return fail(CTQ_ERR_ARG, "null or empty argument");
  *out = nullptr;
  try {
    ctq_impurity* imp = new ctq_impurity();
    ctq::HostModel& h = imp->host;
    h.n_flav = n_flav;
    h.n_sec = n_sec;
    h.is_complex = blocks_im ? 1 : 0;
    h.mu = mu;
    h.dims.assign(dims, dims + n_sec);
    h.N.assign(n_sec, 0);
    if (N) h.N.assign(N, N + n_sec);
    h.E_off.assign(n_sec + 1, 0);
    h.E_min.resize(n_sec);
    h.E_gs = INFINITY;
    for (int q = 0; q < n_sec; ++q) {
      if (dims[q] < 1) { delete imp; return fail(CTQ_ERR_ARG, "sector dimension < 1"); }
      h.E_off[q + 1] = h.E_off[q] + dims[q];
      h.max_dim = std::max(h.max_dim, dims[q]);
    }
    h.E.assign(energies, energies + h.E_off[n_sec]);
    for (int q = 0; q < n_sec; ++q) {
      for (int j = h.E_off[q] + 1; j < h.E_off[q + 1]; ++j)
        if (!(h.E[j] >= h.E[j - 1])) { delete imp; return fail(CTQ_ERR_ARG, "energies not ascending"); }
      h.E_min[q] = h.E[h.E_off[q]];
      h.E_gs = std::min(h.E_gs, h.E_min[q]);
    }
    const int na = 2 * n_flav;
    h.s.assign(s_table, s_table + size_t(na) * n_sec);
    h.blk_off.assign(size_t(na) * n_sec, -1);
    h.opnorm.assign(size_t(na) * n_sec, 0.0);
    int64_t total = 0;
    for (int a = 0; a < na; ++a)
      for (int q = 0; q < n_sec; ++q) {
        const int qp = h.s[size_t(a) * n_sec + q];
        if (qp < -1 || qp >= n_sec) { delete imp; return fail(CTQ_ERR_ARG, "sector table out of range"); }
        if (qp < 0) continue;
        h.blk_off[size_t(a) * n_sec + q] = total;
        total += int64_t(dims[qp]) * dims[q];
      }
    h.blk_re.assign(blocks_re, blocks_re + total);
    if (blocks_im) h.blk_im.assign(blocks_im, blocks_im + total);
    int k = 0;
    for (int a = 0; a < na; ++a)
      for (int q = 0; q < n_sec; ++q) {
        const size_t i = size_t(a) * n_sec + q;
        const int qp = h.s[i];
        if (qp < 0) continue;
        h.opnorm[i] = opnorm ? opnorm[k]
                             : spectral_norm(dims[qp], dims[q], &h.blk_re[h.blk_off[i]],
                                             blocks_im ? &h.blk_im[h.blk_off[i]] : nullptr);
        ++k;
      }
    imp->device = device;
    int st = upload_model(imp);
    if (st != CTQ_OK) {
      delete imp;
      return st;
    }
    *out = imp;
    return CTQ_OK;
  } catch (const std::bad_alloc&) {
    return fail(CTQ_ERR_NOMEM, "host allocation failed");
  } catch (...) {
    return fail(CTQ_ERR_ARG, "unexpected exception");
  }
}

int ctq_add_bulla_operators(ctq_impurity* imp, const double* h_re, const double* h_im) {
  if (!imp) return fail(CTQ_ERR_ARG, "null impurity");
  ctq::HostModel& h = imp->host;
  if (h.n_extra != 0) return fail(CTQ_ERR_ARG, "the Bulla operators are already present");
  const int nf = h.n_flav, ns = h.n_sec;
  try {
    std::vector<ctq::cplx> t(size_t(nf) * nf);
    if (h_re || h_im) {
      for (size_t i = 0; i < t.size(); ++i) t[i] = ctq::cplx(h_re ? h_re[i] : 0.0, h_im ? h_im[i] : 0.0);
    } else if (h.h1.size() == t.size()) {
      t = h.h1;
    } else {
      return fail(CTQ_ERR_ARG, "a loaded impurity needs the one-body matrix h_re / h_im");
    }
    for (const auto& x : t)
      if (!std::isfinite(x.real()) || !std::isfinite(x.imag())) return fail(CTQ_ERR_ARG, "non-finite one-body term");
    if (!h.is_complex)
      for (const auto& x : t)
        if (x.imag() != 0.0) return fail(CTQ_ERR_ARG, "complex one-body term on a real impurity");
    // B_f(q) = F_f(q) o (E_q,n - E_q',m) - sum_j h_fj F_j(q) in the eigenbasis:
    // <m|[c_f, H]|n> = <m|c_f|n> (E_n - E_m) and [c_f, H - U] = sum_j h_fj c_j.
    std::vector<int> s_new(size_t(nf) * ns, -1);
    std::vector<int64_t> off_new(size_t(nf) * ns, -1);
    std::vector<double> norm_new(size_t(nf) * ns, 0.0);
    std::vector<double> re_new, im_new;
    int64_t total = int64_t(h.blk_re.size());
    for (int f = 0; f < nf; ++f)
      for (int q = 0; q < ns; ++q) {
        const int qp = h.s[size_t(2 * f) * ns + q];
        for (int j = 0; j < nf; ++j) {
          const int qj = h.s[size_t(2 * j) * ns + q];
          if (t[size_t(f) * nf + j] != 0.0 && qj >= 0 && qj != qp)
            return fail(CTQ_ERR_UNSUPPORTED, "the one-body term connects sectors that c_f does not");
        }
        if (qp < 0) continue;
        const int r = h.dims[qp], c = h.dims[q];
        const size_t n = size_t(r) * c;
        std::vector<double> br(n, 0.0), bi(n, 0.0);
        const int64_t o = h.blk_off[size_t(2 * f) * ns + q];
        const double* Eq = &h.E[h.E_off[q]];
        const double* Ep = &h.E[h.E_off[qp]];
        for (int m = 0; m < r; ++m)
          for (int k = 0; k < c; ++k) {
            const double de = Eq[k] - Ep[m];
            br[size_t(m) * c + k] = h.blk_re[o + size_t(m) * c + k] * de;
            if (h.is_complex) bi[size_t(m) * c + k] = h.blk_im[o + size_t(m) * c + k] * de;
          }
        for (int j = 0; j < nf; ++j) {
          const ctq::cplx tj = t[size_t(f) * nf + j];
          if (tj == 0.0 || h.s[size_t(2 * j) * ns + q] < 0) continue;
          const int64_t oj = h.blk_off[size_t(2 * j) * ns + q];
          for (size_t i = 0; i < n; ++i) {
            const double fr = h.blk_re[oj + i], fi = h.is_complex ? h.blk_im[oj + i] : 0.0;
            br[i] -= tj.real() * fr - tj.imag() * fi;
            bi[i] -= tj.real() * fi + tj.imag() * fr;
          }
        }
        const size_t idx = size_t(f) * ns + q;
        s_new[idx] = qp;
        off_new[idx] = total;
        // spectral norm by power iteration; above 400 x 400 the Frobenius
        // norm (an upper bound, so the lazy bounds stay valid)
        if (n <= 160000) {
          norm_new[idx] = spectral_norm(r, c, br.data(), h.is_complex ? bi.data() : nullptr);
        } else {
          double fro = 0.0;
          for (size_t i = 0; i < n; ++i) fro += br[i] * br[i] + bi[i] * bi[i];
          norm_new[idx] = std::sqrt(fro) * (1.0 + 1e-12);
        }
        re_new.insert(re_new.end(), br.begin(), br.end());
        if (h.is_complex) im_new.insert(im_new.end(), bi.begin(), bi.end());
        total += int64_t(n);
      }
    h.s.insert(h.s.end(), s_new.begin(), s_new.end());
    h.blk_off.insert(h.blk_off.end(), off_new.begin(), off_new.end());
    h.opnorm.insert(h.opnorm.end(), norm_new.begin(), norm_new.end());
    h.blk_re.insert(h.blk_re.end(), re_new.begin(), re_new.end());
    if (h.is_complex) h.blk_im.insert(h.blk_im.end(), im_new.begin(), im_new.end());
    h.n_extra = nf;
  } catch (const std::bad_alloc&) {
    return fail(CTQ_ERR_NOMEM, "host allocation failed");
  }
  // every device copy (blocks, precision-specific operand formats, launch
  // configurations) is rebuilt for the larger operator table
  free_device(imp);
  imp->dev = ctq::DevModel{};
  imp->launch = ctq::LaunchCfg{};
  imp->rho_off = nullptr;
  imp->tc1 = imp->tc2 = imp->tc3 = ctq::TcParams{};
  imp->launch_tc1 = imp->launch_tc2 = imp->launch_tc3 = ctq::LaunchCfg{};
  imp->big = imp->big64 = false;
  imp->b64 = ctq::Big64Params{};
  imp->launch_b64 = ctq::LaunchCfg{};
  imp->big1 = imp->big2 = imp->big3 = ctq::BigParams{};
  imp->launch_big1 = imp->launch_big2 = imp->launch_big3 = ctq::LaunchCfg{};
  return upload_model(imp);
}

int ctq_impurity_info(const ctq_impurity* imp, ctq_info* out) {
  if (!imp || !out) return fail(CTQ_ERR_ARG, "null argument");
  const ctq::HostModel& h = imp->host;
  out->n_flav = h.n_flav;
  out->n_sec = h.n_sec;
  out->max_dim = h.max_dim;
  out->is_complex = h.is_complex;
  out->mu = h.mu;
  out->E_gs = h.E_gs;
  out->n_block_elems = int64_t(h.blk_re.size());
  out->n_alpha = h.n_alpha();
  return CTQ_OK;
}

int ctq_get_sectors(const ctq_impurity* imp, int* dims, int* N, double* E_min, int* s_table) {
  if (!imp) return fail(CTQ_ERR_ARG, "null impurity");
  const ctq::HostModel& h = imp->host;
  if (dims) std::copy(h.dims.begin(), h.dims.end(), dims);
  if (N) std::copy(h.N.begin(), h.N.end(), N);
  if (E_min) std::copy(h.E_min.begin(), h.E_min.end(), E_min);
  if (s_table) std::copy(h.s.begin(), h.s.begin() + size_t(2 * h.n_flav) * h.n_sec, s_table);
  return CTQ_OK;
}

int ctq_get_energies(const ctq_impurity* imp, int q, double* E) {
  if (!imp || !E || q < 0 || q >= imp->host.n_sec) return fail(CTQ_ERR_ARG, "bad sector");
  const ctq::HostModel& h = imp->host;
  std::copy(h.E.begin() + h.E_off[q], h.E.begin() + h.E_off[q + 1], E);
  return CTQ_OK;
}

int ctq_get_block(const ctq_impurity* imp, int alpha, int q, double* re, double* im) {
  if (!imp || !re) return fail(CTQ_ERR_ARG, "null argument");
  const ctq::HostModel& h = imp->host;
  if (alpha < 0 || alpha >= h.n_alpha() || q < 0 || q >= h.n_sec) return fail(CTQ_ERR_ARG, "bad index");
  const size_t i = size_t(alpha) * h.n_sec + q;
  const int qp = h.s[i];
  if (qp < 0) return fail(CTQ_ERR_ARG, "zero block");
  const size_t cnt = size_t(h.dims[qp]) * h.dims[q];
  const int64_t off = h.blk_off[i];
  std::copy(h.blk_re.begin() + off, h.blk_re.begin() + off + cnt, re);
  if (im) {
    if (h.is_complex)
      std::copy(h.blk_im.begin() + off, h.blk_im.begin() + off + cnt, im);
    else
      std::fill(im, im + cnt, 0.0);
  }
  return CTQ_OK;
}

static int n_seg_of(const ctq_eval_opts* o) {
  const int S = std::max(1, o->segment);
  return (std::max(0, o->max_ops) + S - 1) / S;
}

static size_t big_extra(const ctq_impurity* imp, const ctq_eval_opts* opts) {
  if (opts->precision == CTQ_FP64 || opts->precision == CTQ_F32X2)
    return imp->big64 ? ctq::big64_scratch_bytes(imp->host, std::max(0, opts->max_ops), imp->num_sms) + 256 : 0;
  if (!imp->big) return 0;
  return ctq::big_scratch_bytes(imp->host, std::max(0, opts->max_ops), imp->num_sms) + 256;
}

size_t ctq_workspace_size(const ctq_impurity* imp, int n_chains, const ctq_eval_opts* opts) {
  if (!imp || !opts || n_chains < 0) return 0;
  return ctq::workspace_layout(n_chains, imp->host.n_sec, n_seg_of(opts), nullptr, nullptr) + big_extra(imp, opts);
}

int ctq_launches_per_eval(const ctq_impurity* imp, const ctq_eval_opts* opts) {
  if (!imp || !opts) return 0;
  return 3;  // plan, trace, combine
}

size_t ctq_density_size(const ctq_impurity* imp) {
  if (!imp) return 0;
  return ctq::rho_elems(imp->host) * (imp->host.is_complex ? 2 : 1);
}

size_t ctq_density_workspace_size(const ctq_impurity* imp, int n_chains, const ctq_eval_opts* opts) {
  if (!imp || !opts || n_chains < 0) return 0;
  const size_t base = ctq::workspace_layout(n_chains, imp->host.n_sec, n_seg_of(opts), nullptr, nullptr);
  const int grid = ctq::rho_grid(imp->dev, imp->num_sms, std::max(0, opts->max_ops), ctq_density_size(imp));
  return ((base + 255) & ~size_t(255)) + ctq::rho_scratch_bytes(imp->host, std::max(0, opts->max_ops), grid);
}

int ctq_eval_density_matrices(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                              const ctq_result* result, double* rho, void* workspace, size_t workspace_bytes,
                              void* stream) {
  if (!imp || !batch || !opts || !result || !rho) return fail(CTQ_ERR_ARG, "null argument");
  if (opts->precision != CTQ_FP64 || opts->lazy) return fail(CTQ_ERR_ARG, "the estimator runs in CTQ_FP64 without lazy rejects");
  if (imp->device < 0) return fail(CTQ_ERR_ARG, "impurity has no device copy");
  if (imp->big64) return fail(CTQ_ERR_UNSUPPORTED, "blocks too large for the density-matrix kernel");
  if (batch->n_chains <= 0) return batch->n_chains == 0 ? CTQ_OK : fail(CTQ_ERR_ARG, "n_chains < 0");
  const size_t need = ctq_density_workspace_size(imp, batch->n_chains, opts);
  if (workspace_bytes < need) return fail(CTQ_ERR_WORKSPACE, "workspace smaller than ctq_density_workspace_size()");
  const int n_seg = n_seg_of(opts);
  const size_t base = ctq::workspace_layout(batch->n_chains, imp->host.n_sec, n_seg, nullptr, nullptr);
  int st = ctq_eval_traces(imp, batch, opts, result, workspace, base, stream);
  if (st != CTQ_OK) return st;
  DeviceGuard g(imp->device);
  if (!g.ok()) return fail(CTQ_ERR_CUDA, "cudaSetDevice failed");
  ctq::Work W;
  ctq::workspace_layout(batch->n_chains, imp->host.n_sec, n_seg, workspace, &W);
  ctq::BatchView B{batch->n_chains, batch->beta, batch->offsets, batch->tau, batch->op, batch->log_threshold};
  ctq::EvalCfg cfg;
  cfg.lazy = 0;
  cfg.has_thr = 0;
  cfg.S = opts->segment;
  cfg.n_seg_max = n_seg;
  cfg.max_ops = opts->max_ops;
  ctq::RhoParams P;
  P.rho = rho;
  P.rho_elems = ctq_density_size(imp);
  P.rho_off = imp->rho_off;
  P.scratch = static_cast<char*>(workspace) + ((base + 255) & ~size_t(255));
  P.scratch_elems = size_t(std::max(opts->max_ops, 1) + 1) * imp->host.max_dim * imp->host.max_dim;
  st = ctq::launch_rho(imp->dev, imp->num_sms, imp->optin, B, cfg, W, *result, P,
                       P.rho_elems * size_t(batch->n_chains), stream);
  if (st != CTQ_OK) return fail(st, st == CTQ_ERR_CUDA ? cudaGetErrorString(cudaGetLastError()) : "launch failed");
  return CTQ_OK;
}

size_t ctq_static_ratio_workspace_size(const ctq_impurity* imp, int n_chains, const ctq_eval_opts* opts) {
  if (!imp || !opts || n_chains < 0) return 0;
  const size_t base = ctq::workspace_layout(n_chains, imp->host.n_sec, n_seg_of(opts), nullptr, nullptr);
  const int grid = ctq::rho_grid(imp->dev, imp->num_sms, std::max(0, opts->max_ops), 0);
  return ((base + 255) & ~size_t(255)) + ctq::rho_scratch_bytes(imp->host, std::max(0, opts->max_ops), grid);
}

int ctq_eval_static_ratios(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                           const ctq_result* result, double* h, int n_ops, void* workspace, size_t workspace_bytes,
                           void* stream) {
  if (!imp || !batch || !opts || !result || !h) return fail(CTQ_ERR_ARG, "null argument");
  if (opts->precision != CTQ_FP64 || opts->lazy) return fail(CTQ_ERR_ARG, "the ratios run in CTQ_FP64 without lazy rejects");
  if (imp->device < 0) return fail(CTQ_ERR_ARG, "impurity has no device copy");
  if (imp->host.n_extra < imp->host.n_flav) return fail(CTQ_ERR_ARG, "no Bulla operators (ctq_add_bulla_operators)");
  if (imp->big64) return fail(CTQ_ERR_UNSUPPORTED, "blocks too large for the static-ratio kernel");
  if (n_ops < 0) return fail(CTQ_ERR_ARG, "n_ops < 0");
  if (batch->n_chains <= 0) return batch->n_chains == 0 ? CTQ_OK : fail(CTQ_ERR_ARG, "n_chains < 0");
  const size_t need = ctq_static_ratio_workspace_size(imp, batch->n_chains, opts);
  if (workspace_bytes < need) return fail(CTQ_ERR_WORKSPACE, "workspace smaller than ctq_static_ratio_workspace_size()");
  const int n_seg = n_seg_of(opts);
  const size_t base = ctq::workspace_layout(batch->n_chains, imp->host.n_sec, n_seg, nullptr, nullptr);
  int st = ctq_eval_traces(imp, batch, opts, result, workspace, base, stream);
  if (st != CTQ_OK) return st;
  DeviceGuard g(imp->device);
  if (!g.ok()) return fail(CTQ_ERR_CUDA, "cudaSetDevice failed");
  ctq::Work W;
  ctq::workspace_layout(batch->n_chains, imp->host.n_sec, n_seg, workspace, &W);
  ctq::BatchView B{batch->n_chains, batch->beta, batch->offsets, batch->tau, batch->op, batch->log_threshold};
  ctq::EvalCfg cfg;
  cfg.lazy = 0;
  cfg.has_thr = 0;
  cfg.S = opts->segment;
  cfg.n_seg_max = n_seg;
  cfg.max_ops = opts->max_ops;
  ctq::RhoParams P;
  P.rho = h;
  P.h_len = size_t(n_ops);
  P.scratch = static_cast<char*>(workspace) + ((base + 255) & ~size_t(255));
  P.scratch_elems = size_t(std::max(opts->max_ops, 1) + 1) * imp->host.max_dim * imp->host.max_dim;
  st = ctq::launch_rho(imp->dev, imp->num_sms, imp->optin, B, cfg, W, *result, P, 2 * size_t(n_ops), stream, true);
  if (st != CTQ_OK) return fail(st, st == CTQ_ERR_CUDA ? cudaGetErrorString(cudaGetLastError()) : "launch failed");
  return CTQ_OK;
}

int ctq_trace_kernel(const ctq_impurity* imp, int precision) {
  if (!imp) return CTQ_ERR_ARG;
  if (imp->device < 0) return CTQ_ERR_ARG;
  if (precision == CTQ_FP64) return imp->big64 ? CTQ_KERNEL_FP64_LARGE : CTQ_KERNEL_FP64_SHARED;
  if (precision == CTQ_F32X2)
    return imp->big64 ? CTQ_KERNEL_FP64_LARGE : imp->dev.blk_x2 ? CTQ_KERNEL_FP64_SHARED : CTQ_ERR_UNSUPPORTED;
  if (precision != CTQ_TF32 && precision != CTQ_TF32X3 && precision != CTQ_BF16X3) return CTQ_ERR_UNSUPPORTED;
  if (imp->big) return CTQ_KERNEL_TC_LARGE;
  const ctq::LaunchCfg& lc = precision == CTQ_TF32     ? imp->launch_tc1
                             : precision == CTQ_BF16X3 ? imp->launch_tc2
                                                       : imp->launch_tc3;
  return lc.per_sm >= 1 ? CTQ_KERNEL_TC_SMALL : CTQ_ERR_UNSUPPORTED;
}

int ctq_eval_traces(const ctq_impurity* imp, const ctq_batch* batch, const ctq_eval_opts* opts,
                    const ctq_result* result, void* workspace, size_t workspace_bytes, void* stream) {
  if (!imp || !batch || !opts || !result) return fail(CTQ_ERR_ARG, "null argument");
  if (opts->threads_per_cta < 0 || opts->threads_per_cta > 512 || opts->threads_per_cta % 32 != 0 ||
      opts->ctas_per_sm < 0 || opts->stages < 0 || opts->stages == 1 || opts->tile_order < 0 || opts->tile_order > 3)
    return fail(CTQ_ERR_ARG, "launch tuning out of range");
  if (imp->device < 0) return fail(CTQ_ERR_ARG, "impurity has no device copy");
  if (batch->n_chains < 0) return fail(CTQ_ERR_ARG, "n_chains < 0");
  if (batch->n_chains == 0) return CTQ_OK;
  if (!batch->offsets || !batch->tau || !batch->op) return fail(CTQ_ERR_ARG, "null batch array");
  if (!(batch->beta > 0.0)) return fail(CTQ_ERR_ARG, "beta <= 0");
  if (!result->log_abs || !result->phase || !result->status) return fail(CTQ_ERR_ARG, "null result array");
  if (opts->segment < 1 || opts->max_ops < 0) return fail(CTQ_ERR_ARG, "segment < 1 or max_ops < 0");
  if (opts->lazy && !batch->log_threshold) return fail(CTQ_ERR_ARG, "lazy evaluation needs thresholds");
  if (opts->precision != CTQ_FP64 && opts->precision != CTQ_TF32 && opts->precision != CTQ_TF32X3 &&
      opts->precision != CTQ_BF16X3 && opts->precision != CTQ_F32X2)
    return fail(CTQ_ERR_UNSUPPORTED, "unknown precision");
  const int pr = opts->precision;
  if (pr == CTQ_F32X2 && !imp->dev.blk_x2 && !imp->big64)
    return fail(CTQ_ERR_UNSUPPORTED, "CTQ_F32X2: no float64 kernel serves this impurity");
  const ctq::TcParams& tcp = pr == CTQ_TF32 ? imp->tc1 : pr == CTQ_BF16X3 ? imp->tc2 : imp->tc3;
  const ctq::LaunchCfg& tcl = pr == CTQ_TF32 ? imp->launch_tc1 : pr == CTQ_BF16X3 ? imp->launch_tc2 : imp->launch_tc3;
  if (pr != CTQ_FP64 && pr != CTQ_F32X2 && !imp->big && tcl.per_sm < 1)
    return fail(CTQ_ERR_UNSUPPORTED, "no tensor-core path for this impurity");
  if (!workspace) return fail(CTQ_ERR_ARG, "null workspace");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(CTQ_ERR_ARG, "workspace not 256-byte aligned");
  const int n_seg = n_seg_of(opts);
  const size_t base = ctq::workspace_layout(batch->n_chains, imp->host.n_sec, n_seg, nullptr, nullptr);
  const size_t need = base + big_extra(imp, opts);
  if (workspace_bytes < need) return fail(CTQ_ERR_WORKSPACE, "workspace smaller than ctq_workspace_size()");
  DeviceGuard g(imp->device);
  if (!g.ok()) return fail(CTQ_ERR_CUDA, "cudaSetDevice failed");

  ctq::Work W;
  ctq::workspace_layout(batch->n_chains, imp->host.n_sec, n_seg, workspace, &W);
  ctq::BatchView B{batch->n_chains, batch->beta, batch->offsets, batch->tau, batch->op, batch->log_threshold};
  ctq::EvalCfg cfg;
  cfg.lazy = opts->lazy ? 1 : 0;
  cfg.has_thr = batch->log_threshold ? 1 : 0;
  cfg.S = opts->segment;
  cfg.n_seg_max = n_seg;
  cfg.max_ops = opts->max_ops;
  // Safety margin (log units) before an early reject: float64 rounding, or the
  // relative error of reduced-precision products over a chain.
  // Bounds are norms (no cancellation), so their relative error is about
  // n u for n products: TF32 (u = 2^-11, n <= 400) and 3xTF32 (u ~ 2^-22).
  // BF16X3 keeps 16 significant bits (u ~ 2^-16).
  // CTQ_F32X2 takes the bound's norm from the high float words (relative
  // error ~ 2^-24 per element).
  cfg.margin = opts->precision == CTQ_FP64     ? 1e-9
               : opts->precision == CTQ_F32X2  ? 1e-5
               : opts->precision == CTQ_TF32   ? 0.5
               : opts->precision == CTQ_BF16X3 ? 5e-2
                                               : 1e-2;
  cfg.bounds = result->bounds;
  cfg.debug = opts->debug_flags;
  cfg.threads = opts->threads_per_cta;
  cfg.ctas_per_sm = opts->ctas_per_sm;
  cfg.stages = opts->stages;
  cfg.tile_order = opts->tile_order;
  int st;
  if ((opts->precision == CTQ_FP64 || opts->precision == CTQ_F32X2) && imp->big64) {
    ctq::Big64Params P = imp->b64;
    P.timeout_ns = opts->timeout_ns > 0 ? uint64_t(opts->timeout_ns) : uint64_t(2000000000ull);
    char* scratch = static_cast<char*>(workspace) + ((base + 255) & ~size_t(255));
    st = ctq::launch_eval_big64(imp->dev, imp->launch_b64, P, B, cfg, W, result, scratch, stream,
                                opts->timing_events, opts->precision == CTQ_F32X2);
  } else if (opts->precision == CTQ_FP64 || opts->precision == CTQ_F32X2) {
    st = ctq::launch_eval_fp64(imp->dev, imp->launch, B, cfg, W, result, stream, opts->timing_events,
                               opts->precision == CTQ_F32X2);
  } else if (imp->big) {
    ctq::BigParams P = pr == CTQ_TF32 ? imp->big1 : pr == CTQ_BF16X3 ? imp->big2 : imp->big3;
    const ctq::LaunchCfg& lc = pr == CTQ_TF32 ? imp->launch_big1 : pr == CTQ_BF16X3 ? imp->launch_big2 : imp->launch_big3;
    P.timeout_ns = opts->timeout_ns > 0 ? uint64_t(opts->timeout_ns) : uint64_t(2000000000ull);
    char* scratch = static_cast<char*>(workspace) + ((base + 255) & ~size_t(255));
    st = ctq::launch_eval_big(imp->dev, lc, P, B, cfg, W, result, scratch, stream, opts->timing_events);
  } else {
    ctq::TcParams P = tcp;
    P.timeout_ns = opts->timeout_ns > 0 ? uint64_t(opts->timeout_ns) : uint64_t(2000000000ull);
    st = ctq::launch_eval_tc(imp->dev, tcl, P, B, cfg, W, result, stream, opts->timing_events);
  }
  if (st != CTQ_OK) return fail(st, st == CTQ_ERR_CUDA ? cudaGetErrorString(cudaGetLastError()) : "launch failed");
  return CTQ_OK;
}

int ctq_static_ratios(int m, const int32_t* chain, int n_chains, const double* log_abs, const double* phase,
                      const double* log_abs_u, const double* phase_u, double* h, void* stream) {
  if (m < 0 || n_chains < 0) return fail(CTQ_ERR_ARG, "negative size");
  if (m == 0) return CTQ_OK;
  if (!chain || !log_abs || !phase || !log_abs_u || !phase_u || !h) return fail(CTQ_ERR_ARG, "null pointer");
  const int st = ctq::launch_static_ratios(m, chain, n_chains, log_abs, phase, log_abs_u, phase_u, h, stream);
  return st == CTQ_OK ? CTQ_OK : fail(st, "static-ratio kernel launch failed");
}

void ctq_free_impurity(ctq_impurity* imp) {
  if (!imp) return;
  free_device(imp);
  delete imp;
}

}  // extern "C"
