// Set-up linear algebra for large sectors on the impurity's device: the
// Hermitian eigensolver (cuSOLVER heevd / syevd) and the block transforms
// F = V_{q'}^H C V_q (cuBLAS gemm).  Both libraries are loaded with dlopen the
// first time a sector is too large for the host Jacobi solver, so libctq has
// no link-time dependency on them.  Not on the evaluation path.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cublas_v2.h>
#include <cusolverDn.h>

#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "ctq_internal.h"

namespace ctq {
namespace {

struct DeviceLA {
  bool ok = false;
  std::string err;
  decltype(&cusolverDnCreate) sv_create = nullptr;
  decltype(&cusolverDnDestroy) sv_destroy = nullptr;
  decltype(&cusolverDnZheevd_bufferSize) zheevd_bs = nullptr;
  decltype(&cusolverDnZheevd) zheevd = nullptr;
  decltype(&cusolverDnDsyevd_bufferSize) dsyevd_bs = nullptr;
  decltype(&cusolverDnDsyevd) dsyevd = nullptr;
  decltype(&cublasCreate_v2) bl_create = nullptr;
  decltype(&cublasDestroy_v2) bl_destroy = nullptr;
  decltype(&cublasZgemm_v2) zgemm = nullptr;
  decltype(&cublasDgemm_v2) dgemm = nullptr;
};

// The first of the names (or of $env, if set) that loads; on failure
// *why lists every name tried with the loader's message.
void* open_lib(const char* env, const char* const* names, std::string* why) {
  std::vector<const char*> tries;
  const char* over = std::getenv(env);
  if (over && *over) tries.push_back(over);
  for (int i = 0; names[i]; ++i) tries.push_back(names[i]);
  for (const char* n : tries) {
    void* h = dlopen(n, RTLD_NOW | RTLD_GLOBAL);
    if (h) return h;
    const char* e = dlerror();
    *why += std::string(" [") + n + ": " + (e ? e : "not found") + "]";
  }
  return nullptr;
}

DeviceLA& la() {
  static DeviceLA L;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* sv_names[] = {"libcusolver.so.12", "libcusolver.so", "/usr/local/cuda/lib64/libcusolver.so.12",
                              "/usr/local/cuda/lib64/libcusolver.so", nullptr};
    const char* bl_names[] = {"libcublas.so.13", "libcublas.so", "/usr/local/cuda/lib64/libcublas.so.13",
                              "/usr/local/cuda/lib64/libcublas.so", nullptr};
    std::string why_s, why_b;
    void* hs = open_lib("CTQ_CUSOLVER_LIB", sv_names, &why_s);
    void* hb = open_lib("CTQ_CUBLAS_LIB", bl_names, &why_b);
    if (!hs || !hb) {
      // sectors above kJacobiMaxDim are diagonalised with cuSOLVER (set-up only);
      // CTQ_CUSOLVER_LIB / CTQ_CUBLAS_LIB name the libraries when they are elsewhere
      L.err = "cannot load " + std::string(!hs ? "cuSOLVER" : "cuBLAS") +
              " (needed to diagonalise sectors larger than 160 states; set CTQ_CUSOLVER_LIB / CTQ_CUBLAS_LIB"
              " to the library paths):" + (!hs ? why_s : why_b);
      return;
    }
#define LOAD(h, field, sym) L.field = reinterpret_cast<decltype(L.field)>(dlsym(h, #sym))
    LOAD(hs, sv_create, cusolverDnCreate);
    LOAD(hs, sv_destroy, cusolverDnDestroy);
    LOAD(hs, zheevd_bs, cusolverDnZheevd_bufferSize);
    LOAD(hs, zheevd, cusolverDnZheevd);
    LOAD(hs, dsyevd_bs, cusolverDnDsyevd_bufferSize);
    LOAD(hs, dsyevd, cusolverDnDsyevd);
    LOAD(hb, bl_create, cublasCreate_v2);
    LOAD(hb, bl_destroy, cublasDestroy_v2);
    LOAD(hb, zgemm, cublasZgemm_v2);
    LOAD(hb, dgemm, cublasDgemm_v2);
#undef LOAD
    L.ok = L.sv_create && L.sv_destroy && L.zheevd_bs && L.zheevd && L.dsyevd_bs && L.dsyevd && L.bl_create &&
           L.bl_destroy && L.zgemm && L.dgemm;
    if (!L.ok) L.err = "cuSOLVER / cuBLAS symbols missing";
  });
  return L;
}

// G = C V restricted to the target sector: row k of G is sign * row j of V
// for every (j -> k) pair of the operator; column-major (d_t x d_s).
__global__ void k_gather_rows(const double* V, int cplx, int d_s, const int* src, const int* dst, const double* sg,
                              int n_pairs, int d_t, double* G) {
  const long long total = (long long)n_pairs * d_s;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int p = int(e / d_s), col = int(e - (long long)p * d_s);
    const size_t from = size_t(src[p]) + size_t(col) * d_s;   // V column-major d_s x d_s
    const size_t to = size_t(dst[p]) + size_t(col) * d_t;     // G column-major d_t x d_s
    if (cplx) {
      G[2 * to] = sg[p] * V[2 * from];
      G[2 * to + 1] = sg[p] * V[2 * from + 1];
    } else {
      G[to] = sg[p] * V[from];
    }
  }
}

}  // namespace

struct DeviceSectorLA::Impl {
  int device = -1;
  bool cplx = false;
  cusolverDnHandle_t sv = nullptr;
  cublasHandle_t bl = nullptr;
  std::vector<double*> V;  // per sector: eigenvectors, column-major, on the device (or null)
  std::vector<int> dims;
};

DeviceSectorLA::DeviceSectorLA() : impl_(new Impl) {}

DeviceSectorLA::~DeviceSectorLA() {
  DeviceLA& L = la();
  for (double* p : impl_->V) cudaFree(p);
  if (impl_->sv && L.sv_destroy) L.sv_destroy(impl_->sv);
  if (impl_->bl && L.bl_destroy) L.bl_destroy(impl_->bl);
  delete impl_;
}

int DeviceSectorLA::init(int device, bool cplx, int n_sec, std::string& err) {
  DeviceLA& L = la();
  if (!L.ok) {
    err = L.err;
    return CTQ_ERR_UNSUPPORTED;
  }
  if (device < 0 || cudaSetDevice(device) != cudaSuccess) {
    err = "large sectors need a CUDA device";
    return CTQ_ERR_UNSUPPORTED;
  }
  impl_->device = device;
  impl_->cplx = cplx;
  impl_->V.assign(n_sec, nullptr);
  impl_->dims.assign(n_sec, 0);
  if (L.sv_create(&impl_->sv) != CUSOLVER_STATUS_SUCCESS || L.bl_create(&impl_->bl) != CUBLAS_STATUS_SUCCESS) {
    err = "cannot create cuSOLVER / cuBLAS handles";
    return CTQ_ERR_CUDA;
  }
  return CTQ_OK;
}

// Eigen-decomposition of the Hermitian H (row-major, n x n) on the device.
// A row-major array read as column-major is H^T = conj(H), so the solver
// returns conj(V); E ascending.  V (row-major) is returned to the host and the
// device copy (column-major V) is kept for block transforms.
int DeviceSectorLA::eigh(int q, int n, const std::vector<cplx>& H, std::vector<double>& E, std::vector<cplx>* Vc,
                         std::vector<double>* Vr, std::string& err) {
  DeviceLA& L = la();
  const bool c = impl_->cplx;
  const size_t nn = size_t(n) * n;
  double *dA = nullptr, *dW = nullptr, *dwork = nullptr;
  int* dinfo = nullptr;
  int st = CTQ_OK;
  std::vector<double> hostA(c ? 2 * nn : nn);
  for (size_t i = 0; i < nn; ++i) {
    if (c) {
      hostA[2 * i] = H[i].real();
      hostA[2 * i + 1] = H[i].imag();
    } else {
      hostA[i] = H[i].real();
    }
  }
  if (cudaMalloc(&dA, hostA.size() * 8) || cudaMalloc(&dW, size_t(n) * 8) || cudaMalloc(&dinfo, 4)) {
    err = "device allocation failed";
    st = CTQ_ERR_NOMEM;
  }
  int lwork = 0;
  if (st == CTQ_OK) {
    cudaMemcpy(dA, hostA.data(), hostA.size() * 8, cudaMemcpyHostToDevice);
    cusolverStatus_t s;
    if (c)
      s = L.zheevd_bs(impl_->sv, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                      reinterpret_cast<cuDoubleComplex*>(dA), n, dW, &lwork);
    else
      s = L.dsyevd_bs(impl_->sv, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dW, &lwork);
    if (s != CUSOLVER_STATUS_SUCCESS || cudaMalloc(&dwork, size_t(lwork) * (c ? 16 : 8))) {
      err = "eigensolver workspace";
      st = CTQ_ERR_NOMEM;
    }
  }
  if (st == CTQ_OK) {
    cusolverStatus_t s;
    if (c)
      s = L.zheevd(impl_->sv, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, reinterpret_cast<cuDoubleComplex*>(dA),
                   n, dW, reinterpret_cast<cuDoubleComplex*>(dwork), lwork, dinfo);
    else
      s = L.dsyevd(impl_->sv, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dW, dwork, lwork, dinfo);
    int info = -1;
    cudaMemcpy(&info, dinfo, 4, cudaMemcpyDeviceToHost);
    if (s != CUSOLVER_STATUS_SUCCESS || info != 0) {
      err = "device eigensolver failed";
      st = CTQ_ERR_NUMERIC;
    }
  }
  if (st == CTQ_OK) {
    E.resize(n);
    cudaMemcpy(E.data(), dW, size_t(n) * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(hostA.data(), dA, hostA.size() * 8, cudaMemcpyDeviceToHost);
    // column-major conj(V) -> row-major V; keep column-major V on the device
    for (int col = 0; col < n; ++col)
      for (int row = 0; row < n; ++row) {
        const size_t cm = size_t(row) + size_t(col) * n;
        if (c) {
          const cplx v(hostA[2 * cm], -hostA[2 * cm + 1]);
          (*Vc)[size_t(row) * n + col] = v;
          hostA[2 * cm + 1] = -hostA[2 * cm + 1];
        } else {
          (*Vr)[size_t(row) * n + col] = hostA[cm];
        }
      }
    cudaMemcpy(dA, hostA.data(), hostA.size() * 8, cudaMemcpyHostToDevice);
    impl_->V[q] = dA;
    impl_->dims[q] = n;
    dA = nullptr;
  }
  cudaFree(dA);
  cudaFree(dW);
  cudaFree(dwork);
  cudaFree(dinfo);
  return st;
}

bool DeviceSectorLA::has(int q) const { return impl_->V[q] != nullptr; }

// F = V_{qp}^H (C V_q) for the signed partial permutation C given by pairs
// (source state j, target state k, sign); F is returned row-major
// (d_qp x d_q) into re / im.
int DeviceSectorLA::block(int q, int qp, const std::vector<int>& src, const std::vector<int>& dst,
                          const std::vector<double>& sg, double* re, double* im, std::string& err) {
  DeviceLA& L = la();
  const bool c = impl_->cplx;
  const int ds = impl_->dims[q], dt = impl_->dims[qp];
  const int el = c ? 2 : 1;
  const int np = int(src.size());
  double *dG = nullptr, *dF = nullptr, *dsg = nullptr;
  int *dsrc = nullptr, *ddst = nullptr;
  int st = CTQ_OK;
  if (cudaMalloc(&dG, size_t(dt) * ds * el * 8) || cudaMalloc(&dF, size_t(dt) * ds * el * 8) ||
      cudaMalloc(&dsrc, size_t(np + 1) * 4) || cudaMalloc(&ddst, size_t(np + 1) * 4) ||
      cudaMalloc(&dsg, size_t(np + 1) * 8)) {
    err = "device allocation failed";
    st = CTQ_ERR_NOMEM;
  }
  if (st == CTQ_OK) {
    cudaMemset(dG, 0, size_t(dt) * ds * el * 8);
    cudaMemcpy(dsrc, src.data(), size_t(np) * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(ddst, dst.data(), size_t(np) * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dsg, sg.data(), size_t(np) * 8, cudaMemcpyHostToDevice);
    k_gather_rows<<<1024, 256>>>(impl_->V[q], c ? 1 : 0, ds, dsrc, ddst, dsg, np, dt, dG);
    cublasStatus_t s;
    if (c) {
      const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
      s = L.zgemm(impl_->bl, CUBLAS_OP_C, CUBLAS_OP_N, dt, ds, dt, &one,
                  reinterpret_cast<const cuDoubleComplex*>(impl_->V[qp]), dt, reinterpret_cast<const cuDoubleComplex*>(dG),
                  dt, &zero, reinterpret_cast<cuDoubleComplex*>(dF), dt);
    } else {
      const double one = 1.0, zero = 0.0;
      s = L.dgemm(impl_->bl, CUBLAS_OP_T, CUBLAS_OP_N, dt, ds, dt, &one, impl_->V[qp], dt, dG, dt, &zero, dF, dt);
    }
    if (s != CUBLAS_STATUS_SUCCESS || cudaDeviceSynchronize() != cudaSuccess) {
      err = "device block transform failed";
      st = CTQ_ERR_CUDA;
    }
  }
  if (st == CTQ_OK) {
    std::vector<double> h(size_t(dt) * ds * el);
    cudaMemcpy(h.data(), dF, h.size() * 8, cudaMemcpyDeviceToHost);
    for (int m = 0; m < dt; ++m)
      for (int n = 0; n < ds; ++n) {
        const size_t cm = size_t(m) + size_t(n) * dt, rm = size_t(m) * ds + n;
        re[rm] = h[el * cm];
        if (c) im[rm] = h[2 * cm + 1];
      }
  }
  cudaFree(dG);
  cudaFree(dF);
  cudaFree(dsrc);
  cudaFree(ddst);
  cudaFree(dsg);
  return st;
}

}  // namespace ctq
