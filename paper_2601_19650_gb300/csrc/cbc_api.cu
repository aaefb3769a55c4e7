// C ABI of the CBC library: handles, validation, and the sweep planners that issue
// the kernels of Sec. III A (tensor train) and Sec. III B (trees).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels.cuh"
#include "planner.h"

using namespace cbc;

// ----------------------------------------------------------------------------------
// error reporting
// ----------------------------------------------------------------------------------
static thread_local std::string g_last_error;

int cbc::fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cbc::cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(CBC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(CBC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int cbc::num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

// ----------------------------------------------------------------------------------
// networks
// ----------------------------------------------------------------------------------
static bool valid_dtype(int dt) { return dt == CBC_F32 || dt == CBC_F64 || dt == CBC_C64 || dt == CBC_C128; }
static size_t dtype_bytes(int dt) {
  switch (dt) {
    case CBC_F32: return 4;
    case CBC_F64: return 8;
    case CBC_C64: return 8;
    default: return 16;
  }
}

// Stream-ordered allocations come from a memory pool the library creates for itself on
// each device (never from the device's default pool, which other code in the process may
// use with its own settings).  The sweeps synchronise once per compressed bond and
// allocate per site; with a release threshold of 0 every synchronisation would hand the
// pool's free memory back to the driver and the next allocation would map it again, so
// the library's pool keeps freed memory (release threshold UINT64_MAX).
cudaError_t cbc::pool_malloc(void** p, size_t bytes, cudaStream_t s) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np;
      e = cudaMemPoolCreate(&np, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(np);
        return e;
      }
      pools[dev] = np;
    }
    pool = pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

static int build_network(Net* net, int kind, int n_nodes, const int32_t* parent,
                         const int64_t* phys_dim, const int64_t* bond_dim, int dtype,
                         const void* const* node_data, int data_on_device, void* stream) {
  if (n_nodes < 1 || !parent || !phys_dim || !bond_dim || !node_data)
    return fail(CBC_ERR_INVALID_ARG, "create: null argument or n_nodes < 1");
  if (!valid_dtype(dtype)) return fail(CBC_ERR_INVALID_ARG, "create: bad dtype %d", dtype);
  net->kind = kind;
  net->n = n_nodes;
  net->parent.assign(parent, parent + n_nodes);
  net->phys.assign(phys_dim, phys_dim + n_nodes);
  net->bond.assign(bond_dim, bond_dim + n_nodes);
  net->stream = static_cast<cudaStream_t>(stream);
  net->cplx = (dtype == CBC_C64 || dtype == CBC_C128);
  int roots = 0;
  for (int i = 0; i < n_nodes; ++i) {
    if (parent[i] < -1 || parent[i] >= n_nodes || parent[i] == i)
      return fail(CBC_ERR_INVALID_ARG, "create: parent[%d] = %d invalid", i, parent[i]);
    if (parent[i] < 0) {
      roots++;
      net->root = i;
      net->bond[i] = 1;
    }
    if (phys_dim[i] < 1 || bond_dim[i] < 1)
      return fail(CBC_ERR_INVALID_ARG, "create: node %d has a dimension < 1", i);
    if (!node_data[i]) return fail(CBC_ERR_INVALID_ARG, "create: node_data[%d] is NULL", i);
  }
  if (roots != 1) return fail(CBC_ERR_INVALID_ARG, "create: %d roots (need exactly 1)", roots);
  for (int i = 0; i < n_nodes; ++i) {  // every node reaches the root
    int v = i, steps = 0;
    while (parent[v] >= 0 && steps <= n_nodes) {
      v = parent[v];
      ++steps;
    }
    if (steps > n_nodes) return fail(CBC_ERR_INVALID_ARG, "create: parent array has a cycle");
  }
  net->children.assign(n_nodes, {});
  for (int i = 0; i < n_nodes; ++i)
    if (parent[i] >= 0) net->children[parent[i]].push_back(i);
  net->data.assign(n_nodes, nullptr);
  net->numel.assign(n_nodes, 0);
  cudaStream_t s = net->stream;
  const size_t es = net->elem_bytes(), hs = dtype_bytes(dtype);
  // one allocation for all node tensors (and one staging buffer for host input), node i
  // at element offset off[i] (multiples of 32 elements, so every node starts 256-byte
  // aligned in FP64 storage): a few runtime calls per network instead of five per node
  std::vector<int64_t> off(n_nodes + 1, 0);
  for (int i = 0; i < n_nodes; ++i) {
    int64_t ne = net->bond[i] * net->phys[i] * (kind == 1 ? net->phys[i] : 1);
    for (int c : net->children[i]) ne *= net->bond[c];
    net->numel[i] = ne;
    off[i + 1] = off[i] + (ne + 31) / 32 * 32;
  }
  const int64_t total = off[n_nodes];
  cudaError_t e = pool_malloc(&net->block, total * es, s);
  if (e != cudaSuccess) {
    net->block = nullptr;
    return cuda_fail(e, "create: device allocation");
  }
  for (int i = 0; i < n_nodes; ++i) net->data[i] = static_cast<char*>(net->block) + off[i] * es;
  // the widening pass also flags NaN / Inf entries: such inputs are rejected here, before
  // any sweep runs on them
  int* flag = nullptr;
  e = pool_malloc(reinterpret_cast<void**>(&flag), sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "create: alloc");
  e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "create: memset");
  if (!data_on_device) {
    void* staging = nullptr;
    e = pool_malloc(&staging, total * hs, s);
    if (e != cudaSuccess) return cuda_fail(e, "create: staging alloc");
    // one widening pass over all nodes (the padding between them is zeroed, never read)
    e = cudaMemsetAsync(staging, 0, total * hs, s);
    for (int i = 0; i < n_nodes && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(static_cast<char*>(staging) + off[i] * hs, node_data[i],
                          net->numel[i] * hs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "create: H2D copy");
    e = widen_to_f64(staging, dtype, net->block, total, s, flag);
    if (e != cudaSuccess) return cuda_fail(e, "create: widen");
    cudaFreeAsync(staging, s);
  } else {
    for (int i = 0; i < n_nodes; ++i) {
      e = widen_to_f64(node_data[i], dtype, net->data[i], net->numel[i], s, flag);
      if (e != cudaSuccess) return cuda_fail(e, "create: widen");
    }
  }
  int hflag = 0;
  e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(flag, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "create: synchronize");
  if (hflag) return fail(CBC_ERR_NUMERICAL, "create: a node tensor holds NaN or Inf");
  return CBC_OK;
}

// node tensors are stream-ordered allocations on the network's stream
Net::~Net() {
  bool any = false;
  if (block) {
    cudaFreeAsync(block, stream);
    any = true;
  } else {
    for (void* p : data)
      if (p) {
        cudaFreeAsync(p, stream);
        any = true;
      }
  }
  if (any) cudaStreamSynchronize(stream);
}

struct cbc_ttn_s : Net {};
struct cbc_ttno_s : Net {};

extern "C" {

int ttn_create(int n_nodes, const int32_t* parent, const int64_t* phys_dim,
               const int64_t* bond_dim, int dtype, const void* const* node_data,
               int data_on_device, void* cuda_stream, ttn_t* out) {
  if (!out) return fail(CBC_ERR_INVALID_ARG, "ttn_create: out is NULL");
  *out = nullptr;
  auto* h = new cbc_ttn_s();
  int rc = build_network(h, 0, n_nodes, parent, phys_dim, bond_dim, dtype, node_data,
                         data_on_device, cuda_stream);
  if (rc != CBC_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return CBC_OK;
}

int ttno_create(int n_nodes, const int32_t* parent, const int64_t* phys_dim,
                const int64_t* bond_dim, int dtype, const void* const* node_data,
                int data_on_device, void* cuda_stream, ttno_t* out) {
  if (!out) return fail(CBC_ERR_INVALID_ARG, "ttno_create: out is NULL");
  *out = nullptr;
  auto* h = new cbc_ttno_s();
  int rc = build_network(h, 1, n_nodes, parent, phys_dim, bond_dim, dtype, node_data,
                         data_on_device, cuda_stream);
  if (rc != CBC_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return CBC_OK;
}

int ttn_destroy(ttn_t t) {
  if (t) {
    cudaStreamSynchronize(t->stream);
    delete t;
  }
  return CBC_OK;
}

int ttno_destroy(ttno_t t) {
  if (t) {
    cudaStreamSynchronize(t->stream);
    delete t;
  }
  return CBC_OK;
}

const char* cbc_last_error(void) { return g_last_error.c_str(); }

int ttn_get_info(ttn_t t, int32_t* n_nodes_out, int64_t* bond_dims_out, double* log_norm_out,
                 double* discarded_weight_out) {
  if (!t) return fail(CBC_ERR_INVALID_ARG, "ttn_get_info: NULL handle");
  cudaError_t e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) return cuda_fail(e, "ttn_get_info");
  if (n_nodes_out) *n_nodes_out = t->n;
  if (bond_dims_out)
    for (int i = 0; i < t->n; ++i) bond_dims_out[i] = t->bond[i];
  if (log_norm_out) *log_norm_out = t->log_norm;
  if (discarded_weight_out)
    for (int i = 0; i < t->n; ++i)
      discarded_weight_out[i] = (i < (int)t->discarded.size()) ? t->discarded[i] : 0.0;
  return CBC_OK;
}

int ttn_get_node(ttn_t t, int node, void* dst, int dst_on_device, int dtype) {
  if (!t || !dst) return fail(CBC_ERR_INVALID_ARG, "ttn_get_node: NULL argument");
  if (node < 0 || node >= t->n) return fail(CBC_ERR_INVALID_ARG, "ttn_get_node: node %d out of range", node);
  if (!valid_dtype(dtype)) return fail(CBC_ERR_INVALID_ARG, "ttn_get_node: bad dtype");
  bool want_c = (dtype == CBC_C64 || dtype == CBC_C128);
  if (want_c != t->cplx)
    return fail(CBC_ERR_INVALID_ARG, "ttn_get_node: dtype must be %s for this network",
                t->cplx ? "complex" : "real");
  cudaStream_t s = t->stream;
  int64_t ne = t->numel[node];
  size_t bytes = ne * dtype_bytes(dtype);
  cudaError_t e;
  if (dtype == CBC_F64 || dtype == CBC_C128) {
    e = cudaMemcpyAsync(dst, t->data[node], bytes,
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "ttn_get_node: copy");
  } else {
    void* tmp = dst;
    if (!dst_on_device) {
      e = pool_malloc(&tmp, bytes, s);
      if (e != cudaSuccess) return cuda_fail(e, "ttn_get_node: alloc");
    }
    e = narrow_from_f64(t->data[node], t->cplx, tmp, dtype, ne, s);
    if (e != cudaSuccess) return cuda_fail(e, "ttn_get_node: narrow");
    if (!dst_on_device) {
      e = cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return cuda_fail(e, "ttn_get_node: copy");
      cudaFreeAsync(tmp, s);
    }
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "ttn_get_node: synchronize");
  return CBC_OK;
}

int ttn_get_network(ttn_t t, void* dst, int dst_on_device, int dtype) {
  if (!t || !dst) return fail(CBC_ERR_INVALID_ARG, "ttn_get_network: NULL argument");
  if (!valid_dtype(dtype)) return fail(CBC_ERR_INVALID_ARG, "ttn_get_network: bad dtype");
  bool want_c = (dtype == CBC_C64 || dtype == CBC_C128);
  if (want_c != t->cplx)
    return fail(CBC_ERR_INVALID_ARG, "ttn_get_network: dtype must be %s for this network",
                t->cplx ? "complex" : "real");
  cudaStream_t s = t->stream;
  const size_t hs = dtype_bytes(dtype);
  int64_t total = 0;
  for (int i = 0; i < t->n; ++i) total += t->numel[i];
  // every node into one device buffer (the destination itself when it is on the device),
  // then one copy to the host and one synchronisation
  char* gather = static_cast<char*>(dst);
  cudaError_t e = cudaSuccess;
  if (!dst_on_device) {
    e = pool_malloc(reinterpret_cast<void**>(&gather), total * hs, s);
    if (e != cudaSuccess) return cuda_fail(e, "ttn_get_network: alloc");
  }
  int64_t off = 0;
  for (int i = 0; i < t->n && e == cudaSuccess; ++i) {
    if (dtype == CBC_F64 || dtype == CBC_C128)
      e = cudaMemcpyAsync(gather + off * hs, t->data[i], t->numel[i] * hs,
                          cudaMemcpyDeviceToDevice, s);
    else
      e = narrow_from_f64(t->data[i], t->cplx, gather + off * hs, dtype, t->numel[i], s);
    off += t->numel[i];
  }
  if (e == cudaSuccess && !dst_on_device)
    e = cudaMemcpyAsync(dst, gather, total * hs, cudaMemcpyDeviceToHost, s);
  if (!dst_on_device) cudaFreeAsync(gather, s);
  if (e != cudaSuccess) return cuda_fail(e, "ttn_get_network: copy");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "ttn_get_network: synchronize");
  return CBC_OK;
}

static int parse_options(const cbc_options* opt, Options* o) {
  if (opt) {
    o->precision = opt->precision;
    if (opt->slices_fwd > 0) o->slices_fwd = opt->slices_fwd;
    if (opt->slices_bwd > 0) o->slices_bwd = opt->slices_bwd;
    if (opt->max_group < 0 || opt->max_group > 1024)
      return fail(CBC_ERR_INVALID_ARG, "cbc_apply: max_group %d outside [0, 1024]", opt->max_group);
    if (opt->max_group > 0) o->max_group = opt->max_group;
  }
  if (o->precision != CBC_PREC_FP64 && o->precision != CBC_PREC_MIXED)
    return fail(CBC_ERR_INVALID_ARG, "cbc_apply: bad precision %d", o->precision);
  o->eps_rank = (o->precision == CBC_PREC_MIXED) ? 1e-9 : 1e-12;
  if (opt && opt->eps_rank > 0) o->eps_rank = opt->eps_rank;
  return CBC_OK;
}

static int apply_one(ttn_t state, ttno_t op, int64_t max_bond, double tol,
                     const cbc_options* opt, bool concurrent, ttn_t* out);

int cbc_apply(ttn_t state, ttno_t op, int64_t max_bond, double tol, const cbc_options* opt,
              ttn_t* out) {
  return apply_one(state, op, max_bond, tol, opt, false, out);
}

static int apply_one(ttn_t state, ttno_t op, int64_t max_bond, double tol,
                     const cbc_options* opt, bool concurrent, ttn_t* out) {
  if (!out) return fail(CBC_ERR_INVALID_ARG, "cbc_apply: out is NULL");
  *out = nullptr;
  if (!state || !op) return fail(CBC_ERR_INVALID_ARG, "cbc_apply: NULL network");
  if (state->kind != 0 || op->kind != 1) return fail(CBC_ERR_INVALID_ARG, "cbc_apply: wrong handle kinds");
  if (state->n != op->n || state->parent != op->parent || state->phys != op->phys)
    return fail(CBC_ERR_TOPOLOGY_MISMATCH, "cbc_apply: state and operator trees differ");
  if (!std::isfinite(tol)) return fail(CBC_ERR_INVALID_ARG, "cbc_apply: tol is not finite");
  Options o;
  int prc = parse_options(opt, &o);
  if (prc != CBC_OK) return prc;
  o.concurrent = concurrent;
  auto* res = new cbc_ttn_s();
  int rc = run_cbc(*state, *op, max_bond, tol, o, res);
  if (rc != CBC_OK) {
    delete res;
    return rc;
  }
  *out = res;
  return CBC_OK;
}

// ---- comparison methods of Sec. III C on tensor trains --------------------------------
static int check_chain_pair(ttn_t state, ttno_t op, const char* who) {
  if (!state || !op) return fail(CBC_ERR_INVALID_ARG, "%s: NULL network", who);
  if (state->kind != 0 || op->kind != 1) return fail(CBC_ERR_INVALID_ARG, "%s: wrong handle kinds", who);
  if (state->n != op->n || state->parent != op->parent || state->phys != op->phys)
    return fail(CBC_ERR_TOPOLOGY_MISMATCH, "%s: state and operator trees differ", who);
  for (int i = 0; i < state->n; ++i)
    if (state->parent[i] != i - 1)
      return fail(CBC_ERR_UNSUPPORTED, "%s: only tensor trains (parent[i] = i - 1) are supported", who);
  return CBC_OK;
}

static int run_method(ttn_t state, ttno_t op, int64_t max_bond, double tol, Options& o,
                      ttn_t* out) {
  auto* res = new cbc_ttn_s();
  int rc = run_cbc(*state, *op, max_bond, tol, o, res);
  if (rc != CBC_OK) {
    delete res;
    return rc;
  }
  *out = res;
  return CBC_OK;
}

int zipup_apply(ttn_t state, ttno_t op, int64_t max_bond, double tol, const cbc_options* opt,
                ttn_t* out) {
  if (!out) return fail(CBC_ERR_INVALID_ARG, "zipup_apply: out is NULL");
  *out = nullptr;
  int rc = check_chain_pair(state, op, "zipup_apply");
  if (rc != CBC_OK) return rc;
  if (!std::isfinite(tol)) return fail(CBC_ERR_INVALID_ARG, "zipup_apply: tol is not finite");
  Options o;
  rc = parse_options(opt, &o);
  if (rc != CBC_OK) return rc;
  o.method = kMethodZipUp;
  return run_method(state, op, max_bond, tol, o, out);
}

int direct_apply(ttn_t state, ttno_t op, int64_t max_bond, double tol, const cbc_options* opt,
                 ttn_t* out) {
  if (!out) return fail(CBC_ERR_INVALID_ARG, "direct_apply: out is NULL");
  *out = nullptr;
  int rc = check_chain_pair(state, op, "direct_apply");
  if (rc != CBC_OK) return rc;
  if (!std::isfinite(tol)) return fail(CBC_ERR_INVALID_ARG, "direct_apply: tol is not finite");
  Options o;
  rc = parse_options(opt, &o);
  if (rc != CBC_OK) return rc;
  o.method = kMethodDirect;
  return run_method(state, op, max_bond, tol, o, out);
}

int src_apply(ttn_t state, ttno_t op, int64_t sketch_size, const void* const* omega,
              int omega_dtype, int omega_on_device, const cbc_options* opt, ttn_t* out) {
  if (!out) return fail(CBC_ERR_INVALID_ARG, "src_apply: out is NULL");
  *out = nullptr;
  int rc = check_chain_pair(state, op, "src_apply");
  if (rc != CBC_OK) return rc;
  if (sketch_size < 1 || sketch_size > (1 << 20))
    return fail(CBC_ERR_INVALID_ARG, "src_apply: sketch_size %lld outside [1, 2^20]",
                (long long)sketch_size);
  if (!omega || !valid_dtype(omega_dtype))
    return fail(CBC_ERR_INVALID_ARG, "src_apply: omega is NULL or its dtype is invalid");
  const bool ocplx = (omega_dtype == CBC_C64 || omega_dtype == CBC_C128);
  if (ocplx != state->cplx)
    return fail(CBC_ERR_INVALID_ARG,
                "src_apply: omega must be real for real networks and complex for complex ones");
  const int L = state->n;
  for (int i = 0; i + 1 < L; ++i)
    if (!omega[i]) return fail(CBC_ERR_INVALID_ARG, "src_apply: omega[%d] is NULL", i);
  Options o;
  rc = parse_options(opt, &o);
  if (rc != CBC_OK) return rc;
  // the random matrices in FP64 storage of the network's type, one allocation
  cudaStream_t s = state->stream;
  const size_t es = state->elem_bytes(), hs = dtype_bytes(omega_dtype);
  std::vector<int64_t> off(L + 1, 0);
  for (int i = 0; i < L; ++i)
    off[i + 1] = off[i] + ((i + 1 < L) ? (state->phys[i] * sketch_size + 31) / 32 * 32 : 0);
  void* block = nullptr;
  void* flag = nullptr;
  cudaError_t e = pool_malloc(&block, std::max<int64_t>(off[L], 1) * es, s);
  if (e != cudaSuccess) return cuda_fail(e, "src_apply: device allocation");
  std::vector<void*> mats(L, nullptr);
  for (int i = 0; i + 1 < L; ++i) mats[i] = static_cast<char*>(block) + off[i] * es;
  e = pool_malloc(&flag, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  void* staging = nullptr;
  if (e == cudaSuccess && !omega_on_device) {
    e = pool_malloc(&staging, std::max<int64_t>(off[L], 1) * hs, s);
    for (int i = 0; i + 1 < L && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(static_cast<char*>(staging) + off[i] * hs, omega[i],
                          state->phys[i] * sketch_size * hs, cudaMemcpyHostToDevice, s);
  }
  for (int i = 0; i + 1 < L && e == cudaSuccess; ++i)
    e = widen_to_f64(omega_on_device ? omega[i] : static_cast<char*>(staging) + off[i] * hs,
                     omega_dtype, mats[i], state->phys[i] * sketch_size, s,
                     static_cast<int*>(flag));
  int hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (staging) cudaFreeAsync(staging, s);
  if (flag) cudaFreeAsync(flag, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || hflag) {
    cudaFreeAsync(block, s);
    cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "src_apply: upload of omega");
    return fail(CBC_ERR_NUMERICAL, "src_apply: omega holds NaN or Inf");
  }
  o.method = kMethodSRC;
  o.sketch = (int)sketch_size;
  o.sketch_mats = mats.data();
  rc = run_method(state, op, 0, 0.0, o, out);
  cudaFreeAsync(block, s);
  cudaStreamSynchronize(s);
  return rc;
}

int cbc_rank_rule(int n, const double* w, double beyond, int64_t max_bond, double tol,
                  double floor_rel, int* k_out, double* discarded_out) {
  if (n < 1 || !w || !k_out) return fail(CBC_ERR_INVALID_ARG, "cbc_rank_rule: bad arguments");
  if (!std::isfinite(tol) || !std::isfinite(beyond) || !std::isfinite(floor_rel))
    return fail(CBC_ERR_INVALID_ARG, "cbc_rank_rule: non-finite argument");
  const int k = pick_rank(w, n, beyond, max_bond, tol, floor_rel);
  *k_out = k;
  if (discarded_out) {  // (beyond + sum_{j>=k} w_j) / (beyond + sum_j w_j)
    double tail = std::max(beyond, 0.0), total = tail;
    for (int j = 0; j < n; ++j) {
      total += std::max(w[j], 0.0);
      if (j >= k) tail += std::max(w[j], 0.0);
    }
    *discarded_out = (total > 0.0) ? tail / total : 0.0;
  }
  return CBC_OK;
}

int cbc_apply_batched(int n, const ttn_t* states, const ttno_t* ops, const int64_t* max_bond,
                      const double* tol, const cbc_options* opt, int workers, ttn_t* outs) {
  if (n < 0 || (n > 0 && (!states || !ops || !outs)))
    return fail(CBC_ERR_INVALID_ARG, "cbc_apply_batched: bad arguments");
  for (int j = 0; j < n; ++j) outs[j] = nullptr;
  if (n == 0) return CBC_OK;
  // groups: chains with identical shapes, max_bond and tol (at most kMaxGroup each) run
  // in lockstep, one launch per step for the whole group; the rest one by one
  int kMaxGroup = 32;
  {
    Options o;
    if (parse_options(opt, &o) == CBC_OK) kMaxGroup = o.max_group;
  }
  std::vector<std::vector<int>> tasks;
  {
    std::vector<int> open_task;  // index into tasks of the open group per signature
    std::vector<int> leader;     // first member of each open group
    for (int j = 0; j < n; ++j) {
      const ttn_t st = states[j];
      const ttno_t op = ops[j];
      int home = -1;
      if (st && op && st->kind == 0 && op->kind == 1)
        for (size_t q = 0; q < leader.size(); ++q) {
          const int l = leader[q];
          const ttn_t s2 = states[l];
          const ttno_t o2 = ops[l];
          if (tasks[open_task[q]].size() < (size_t)kMaxGroup && s2->cplx == st->cplx &&
              s2->n == st->n && s2->parent == st->parent && s2->phys == st->phys &&
              s2->bond == st->bond && o2->bond == op->bond && o2->parent == op->parent &&
              o2->phys == op->phys && (max_bond ? max_bond[l] == max_bond[j] : true) &&
              (tol ? tol[l] == tol[j] : true)) {
            home = open_task[q];
            break;
          }
        }
      if (home < 0) {
        tasks.push_back({j});
        if (st && op && st->kind == 0 && op->kind == 1) {
          leader.push_back(j);
          open_task.push_back((int)tasks.size() - 1);
        }
      } else {
        tasks[home].push_back(j);
      }
    }
  }
  const int nt = (int)tasks.size();
  if (workers <= 0) workers = std::min(nt, 16);
  workers = std::max(1, std::min(workers, nt));
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int> rc(n, CBC_OK);
  std::vector<std::string> msg(n);
  const bool concurrent = workers > 1;
  auto one = [&](int j) {
    rc[j] = apply_one(states[j], ops[j], max_bond ? max_bond[j] : 0, tol ? tol[j] : 0.0, opt,
                      concurrent, &outs[j]);
    if (rc[j] != CBC_OK) msg[j] = g_last_error;
  };
  auto group = [&](const std::vector<int>& t) {
    const int j0 = t[0];
    Options o;
    int prc = parse_options(opt, &o);
    if (prc == CBC_OK && !std::isfinite(tol ? tol[j0] : 0.0))
      prc = fail(CBC_ERR_INVALID_ARG, "cbc_apply: tol is not finite");
    if (prc != CBC_OK) {
      for (int j : t) {
        rc[j] = prc;
        msg[j] = g_last_error;
      }
      return;
    }
    std::vector<const Net*> sv, ov;
    std::vector<Net*> res;
    for (int j : t) {
      sv.push_back(states[j]);
      ov.push_back(ops[j]);
      res.push_back(new cbc_ttn_s());
    }
    const int grc = run_cbc_group(sv, ov, max_bond ? max_bond[j0] : 0, tol ? tol[j0] : 0.0, o, res);
    if (grc == CBC_OK) {
      for (size_t q = 0; q < t.size(); ++q) outs[t[q]] = static_cast<ttn_t>(res[q]);
      return;
    }
    for (Net* r : res) delete r;
    if (grc == kGroupSplit) {  // members chose different ranks: one by one
      for (int j : t) one(j);
      return;
    }
    for (int j : t) {
      rc[j] = grc;
      msg[j] = g_last_error;
    }
  };
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    for (int q = next++; q < nt; q = next++) {
      if (tasks[q].size() == 1)
        one(tasks[q][0]);
      else
        group(tasks[q]);
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  for (int j = 0; j < n; ++j)
    if (rc[j] != CBC_OK) return fail(rc[j], "cbc_apply_batched: instance %d: %s", j, msg[j].c_str());
  return CBC_OK;
}

int cbc_gemm(int precision, int slices, int dtype, int M, int N, int K, const void* A,
             int64_t lda, int transA, int conjA, const void* B, int64_t ldb, int transB,
             int conjB, void* C, int64_t ldc, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || ldc < N)
    return fail(CBC_ERR_INVALID_ARG, "cbc_gemm: bad arguments");
  if (dtype != CBC_F64 && dtype != CBC_C128)
    return fail(CBC_ERR_INVALID_ARG, "cbc_gemm: dtype must be CBC_F64 or CBC_C128");
  if (precision != CBC_PREC_FP64 && precision != CBC_PREC_MIXED)
    return fail(CBC_ERR_INVALID_ARG, "cbc_gemm: bad precision");
  if (slices == 0) slices = 4;
  if (precision == CBC_PREC_MIXED && (slices < 2 || slices > 5))
    return fail(CBC_ERR_INVALID_ARG, "cbc_gemm: slices must be in [2, 5]");
  View va = transA ? View::transposed(lda) : View::rowmajor(lda);
  View vb = transB ? View::transposed(ldb) : View::rowmajor(ldb);
  View vc = View::rowmajor(ldc);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = nullptr;
  cudaError_t e = pool_malloc(reinterpret_cast<void**>(&status), sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_gemm: alloc");
  e = cudaMemsetAsync(status, 0, sizeof(int), s);
  void* ws = nullptr;
  const bool cplx = dtype == CBC_C128;
  if (e == cudaSuccess && precision == CBC_PREC_MIXED) {
    e = pool_malloc(&ws, gemm_tc_workspace_bytes(M, N, K, cplx, slices), s);
    if (e == cudaSuccess) {
      e = cplx ? gemm_tc<zdbl>(M, N, K, (const zdbl*)A, va, conjA, (const zdbl*)B, vb, conjB,
                               (zdbl*)C, vc, slices, ws, status, s)
               : gemm_tc<double>(M, N, K, (const double*)A, va, conjA, (const double*)B, vb,
                                 conjB, (double*)C, vc, slices, ws, status, s);
    }
  } else if (e == cudaSuccess) {
    e = cplx ? gemm_f64<zdbl>(M, N, K, 1, (const zdbl*)A, va, conjA, (const zdbl*)B, vb, conjB,
                              (zdbl*)C, vc, s)
             : gemm_f64<double>(M, N, K, 1, (const double*)A, va, conjA, (const double*)B, vb,
                                conjB, (double*)C, vc, s);
  }
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ws) cudaFreeAsync(ws, s);
  cudaFreeAsync(status, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_gemm");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cbc_gemm: synchronize");
  if (hs != 0) return fail(hs, "cbc_gemm: device status %d", hs);
  return CBC_OK;
}

}  // extern "C"
