// Host side of the C ABI declared in include/ccz4.h: grid allocation and
// validation, host <-> device copies, and the orchestration of halo fill,
// right-hand side, RK4 stages and constraint monitors. Every compute step
// runs in the kernels of halo.cu, rhs.cu and constraints.cu.
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "ccz4_internal.cuh"
#include "mesh_plan.h"

namespace ccz4 {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int constraint_blocks(long long n_points);
// shared-memory limits of the two-phase stage kernels (rhs_shapes.cu, rhs_mesh_shapes.cu)
cudaError_t prepare_shaped_uniform();
cudaError_t prepare_shaped_mesh();
// constraint norms over the leaf points outside n_centres balls (constraints.cu)
cudaError_t launch_constraints_excluded(const GridView &g, const double *H, const double *M, int n_centres,
                                        const double *centres, double radius, double *partial, int blocks,
                                        double *out5, cudaStream_t s);

}  // namespace ccz4

using namespace ccz4;

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return CCZ4_ERR_CUDA;                                                              \
    }                                                                                    \
  } while (0)

static bool state_buffer(int buf) { return buf >= CCZ4_BUF_U && buf <= CCZ4_BUF_INI; }

static ccz4_status check_grid(const ccz4_grid *g) {
  if (!g) {
    set_error("grid is NULL");
    return CCZ4_ERR_INVALID;
  }
  return CCZ4_OK;
}

static ccz4_status check_params(const ccz4_params *P) {
  if (!P) {
    set_error("params is NULL");
    return CCZ4_ERR_INVALID;
  }
  if (P->slicing != CCZ4_SLICING_HARMONIC && P->slicing != CCZ4_SLICING_ONE_PLUS_LOG) {
    set_error("unknown slicing %d", P->slicing);
    return CCZ4_ERR_INVALID;
  }
  if (P->shift != CCZ4_SHIFT_ZERO && P->shift != CCZ4_SHIFT_GAMMA_DRIVER) {
    set_error("unknown shift condition %d", P->shift);
    return CCZ4_ERR_INVALID;
  }
  if (P->precision != CCZ4_PREC_FP64 && P->precision != CCZ4_PREC_MIXED) {
    set_error("unknown precision %d", P->precision);
    return CCZ4_ERR_INVALID;
  }
  if (!(P->tau != 0.0)) {
    set_error("tau must be non-zero");
    return CCZ4_ERR_INVALID;
  }
  return CCZ4_OK;
}

// The allocator of the large buffers of grids created from now on (ccz4_set_allocator).
static ccz4_alloc_fn g_alloc = nullptr;
static ccz4_dealloc_fn g_dealloc = nullptr;
static void *g_alloc_ctx = nullptr;

extern "C" ccz4_status ccz4_set_allocator(ccz4_alloc_fn alloc, ccz4_dealloc_fn dealloc, void *ctx) {
  if ((alloc == nullptr) != (dealloc == nullptr)) {
    set_error("set_allocator: give both functions or neither");
    return CCZ4_ERR_INVALID;
  }
  g_alloc = alloc;
  g_dealloc = dealloc;
  g_alloc_ctx = alloc ? ctx : nullptr;
  return CCZ4_OK;
}

static void free_all(ccz4_grid *g) {
  if (g->step_exec) cudaGraphExecDestroy(g->step_exec);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  for (int b = 0; b < 8; ++b) {
    if (!g->buf[b]) continue;
    if (g->dealloc)
      g->dealloc(g->alloc_ctx, g->buf[b], sizeof(double) * (size_t)g->buf_len[b], nullptr);
    else
      cudaFree(g->buf[b]);
  }
  cudaFree(g->d_ijk);
  cudaFree(g->d_owner);
  cudaFree(g->d_gcoord);
  cudaFree(g->d_ghost_geo);
  cudaFree(g->d_status);
  cudaFree(g->red_partial);
  cudaFree(g->red_out);
  cudaFreeHost(g->host_out);
  cudaFree(g->d_src);
  cudaFree(g->d_interp);
  cudaFree(g->d_ibeg);
  cudaFree(g->d_xjob);
  cudaFree(g->d_yjob);
  cudaFree(g->d_zjob);
  cudaFree(g->d_xbeg);
  cudaFree(g->d_ybeg);
  cudaFree(g->d_plev);
  cudaFree(g->d_leaf);
  for (int l = 0; l < CCZ4_MAX_LEVELS; ++l) {
    cudaFree(g->d_rpar[l]);
    cudaFree(g->d_rkid[l]);
  }
  cudaFree(g->d_queue);
  free(g);
}

static ccz4_status create_grid(const ccz4_grid_desc *d, const std::vector<int> &owner, const MeshPlan *mesh,
                               ccz4_grid **out);

extern "C" ccz4_status ccz4_alloc_patches(const ccz4_grid_desc *d, ccz4_grid **out) {
  if (!out) {
    set_error("out is NULL");
    return CCZ4_ERR_INVALID;
  }
  *out = nullptr;
  if (!d) {
    set_error("descriptor is NULL");
    return CCZ4_ERR_INVALID;
  }
  if (d->p < 1 || d->np[0] < 1 || d->np[1] < 1 || d->np[2] < 1 || !(d->dx > 0.0)) {
    set_error("invalid sizes: p=%d np=(%d,%d,%d) dx=%g", d->p, d->np[0], d->np[1], d->np[2], d->dx);
    return CCZ4_ERR_INVALID;
  }
  if (d->p > MAX_P) {
    set_error("patch edge p=%d exceeds %d: the halo'd tile of one field must fit in shared memory", d->p, MAX_P);
    return CCZ4_ERR_INVALID;
  }
  if (d->bc != CCZ4_BC_PERIODIC && d->bc != CCZ4_BC_COPY && d->bc != CCZ4_BC_SOMMERFELD) {
    set_error("unknown boundary kind %d", d->bc);
    return CCZ4_ERR_INVALID;
  }
  const long long slots = (long long)d->np[0] * d->np[1] * d->np[2];
  if (slots != d->n_patches || !d->ijk) {
    set_error("n_patches (%d) must equal np0*np1*np2 (%lld) and ijk must be given", d->n_patches, slots);
    return CCZ4_ERR_INVALID;
  }
  const long long Nx = (long long)d->np[0] * d->p, Ny = (long long)d->np[1] * d->p, Nz = (long long)d->np[2] * d->p;
  if (Nx + 2 * HALO > (1 << 30) || Ny + 2 * HALO > (1 << 30) || Nz + 2 * HALO > (1 << 30)) {
    set_error("domain too large for 32-bit point coordinates");
    return CCZ4_ERR_INVALID;
  }
  std::vector<int> owner((size_t)slots, -1);
  for (int n = 0; n < d->n_patches; ++n) {
    const int a = d->ijk[3 * n], b = d->ijk[3 * n + 1], c = d->ijk[3 * n + 2];
    if (a < 0 || a >= d->np[0] || b < 0 || b >= d->np[1] || c < 0 || c >= d->np[2]) {
      set_error("patch %d has coordinates (%d,%d,%d) outside the %dx%dx%d block", n, a, b, c, d->np[0],
                d->np[1], d->np[2]);
      return CCZ4_ERR_INVALID;
    }
    const long long cell = ((long long)c * d->np[1] + b) * d->np[0] + a;
    if (owner[cell] >= 0) {
      set_error("patch slot (%d,%d,%d) is listed twice", a, b, c);
      return CCZ4_ERR_INVALID;
    }
    owner[cell] = n;
  }
  return create_grid(d, owner, nullptr, out);
}

extern "C" ccz4_status ccz4_alloc_mesh(const ccz4_mesh_desc *m, ccz4_grid **out) {
  if (!out) {
    set_error("out is NULL");
    return CCZ4_ERR_INVALID;
  }
  *out = nullptr;
  MeshPlan plan;
  ccz4_status st = plan_mesh(m, true, plan);
  if (st != CCZ4_OK) return st;
  // separable coarse-to-fine interpolation unless CCZ4_MESH_INTERP_BY_ENTRY=1
  const char *by_entry = getenv("CCZ4_MESH_INTERP_BY_ENTRY");
  const long long T = m->p + 2 * HALO;
  plan_separable(plan, (by_entry && by_entry[0] == '1') ? 0 : T * T * T);
  ccz4_grid_desc d;
  d.p = m->p;
  d.n_patches = m->n_patches;
  d.ijk = m->ijk;
  for (int q = 0; q < 3; ++q) {
    d.np[q] = m->np[q];
    d.origin[q] = m->origin[q];
  }
  d.dx = m->dx;
  d.bc = m->bc;
  return create_grid(&d, plan.owner0, &plan, out);
}

template <class T>
static bool upload_table(T **dst, const T *src, size_t n) {
  if (n == 0) return true;
  if (cudaMalloc(dst, sizeof(T) * n) != cudaSuccess) return false;
  return cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice) == cudaSuccess;
}

// Builds the device grid of a validated descriptor: level-0 slot owners in
// `owner`; `mesh` holds the tables of a refined mesh, or is NULL.
static ccz4_status create_grid(const ccz4_grid_desc *d, const std::vector<int> &owner, const MeshPlan *mesh,
                               ccz4_grid **out) {
  const long long slots = (long long)d->np[0] * d->np[1] * d->np[2];
  const long long Nx = (long long)d->np[0] * d->p, Ny = (long long)d->np[1] * d->p, Nz = (long long)d->np[2] * d->p;
  ccz4_grid *g = (ccz4_grid *)calloc(1, sizeof(ccz4_grid));
  if (!g) {
    set_error("host allocation failed");
    return CCZ4_ERR_NOMEM;
  }
  GridView &v = g->v;
  v.p = d->p;
  v.T = d->p + 2 * HALO;
  for (int q = 0; q < 3; ++q) {
    v.np[q] = d->np[q];
    v.origin[q] = d->origin[q];
  }
  v.N[0] = (int)Nx;
  v.N[1] = (int)Ny;
  v.N[2] = (int)Nz;
  v.n_patches = d->n_patches;
  v.bc = d->bc;
  v.dx = d->dx;
  v.n_points = (long long)d->n_patches * d->p * d->p * d->p;
  v.T3 = (long long)v.T * v.T * v.T;
  v.n_levels = mesh ? mesh->n_levels : 1;
  v.n_leaf_points = mesh ? mesh->n_leaf_points : v.n_points;
  v.ldx[0] = d->dx;
  for (int l = 1; l < MAX_LEVELS; ++l) v.ldx[l] = v.ldx[l - 1] / 3.0;
  std::vector<int> gcoord;
  if (d->bc == CCZ4_BC_SOMMERFELD) {
    v.n_ghost = (Nx + 6) * (Ny + 6) * (Nz + 6) - Nx * Ny * Nz;
    gcoord.reserve((size_t)(3 * v.n_ghost));
    for (int z = -HALO; z < Nz + HALO; ++z)
      for (int y = -HALO; y < Ny + HALO; ++y)
        for (int x = -HALO; x < Nx + HALO; ++x) {
          if (x >= 0 && x < Nx && y >= 0 && y < Ny && z >= 0 && z < Nz) {
            x = (int)Nx - 1;  // jump over the interior of this row
            continue;
          }
          gcoord.push_back(x);
          gcoord.push_back(y);
          gcoord.push_back(z);
        }
  } else {
    v.n_ghost = 0;
  }
  v.S = ((v.n_points + v.n_ghost + 31) / 32) * 32;
  if (v.S == 0) v.S = 32;
  if (v.S > 0x7FFFFFFFLL) {
    set_error("grid too large: %lld points per field exceed 32-bit indexing", v.S);
    free(g);
    return CCZ4_ERR_INVALID;
  }
  cudaGetDevice(&g->device);
  const long long state_len = (long long)NV * v.S;
  const long long lens[8] = {state_len, state_len, state_len, state_len, state_len,
                             d->bc == CCZ4_BC_SOMMERFELD ? state_len : 0,
                             (long long)NV * v.n_patches * v.T3, (long long)NMIX * v.n_points};
  g->alloc = g_alloc;
  g->dealloc = g_dealloc;
  g->alloc_ctx = g_alloc_ctx;
  for (int b = 0; b < 8; ++b) {
    g->buf_len[b] = lens[b];
    if (lens[b] == 0) continue;
    const size_t bytes = sizeof(double) * (size_t)lens[b];
    if (g->alloc) {
      g->buf[b] = (double *)g->alloc(g->alloc_ctx, bytes, nullptr);
      if (!g->buf[b] || ((uintptr_t)g->buf[b] & 255u)) {
        set_error("the allocator returned %s for %zu bytes", g->buf[b] ? "an unaligned pointer" : "NULL", bytes);
        if (g->buf[b]) {
          g->dealloc(g->alloc_ctx, g->buf[b], bytes, nullptr);
          g->buf[b] = nullptr;
        }
        free_all(g);
        return CCZ4_ERR_NOMEM;
      }
    } else {
      cudaError_t e = cudaMalloc(&g->buf[b], bytes);
      if (e != cudaSuccess) {
        g->buf[b] = nullptr;
        set_error("cudaMalloc of %lld doubles failed: %s", lens[b], cudaGetErrorString(e));
        cudaGetLastError();
        free_all(g);
        return CCZ4_ERR_NOMEM;
      }
    }
    cudaMemset(g->buf[b], 0, bytes);
  }
  g->red_blocks = constraint_blocks(v.n_points);
  bool ok = cudaMalloc(&g->d_ijk, sizeof(int) * 3 * (size_t)d->n_patches) == cudaSuccess &&
            cudaMalloc(&g->d_owner, sizeof(int) * (size_t)slots) == cudaSuccess &&
            cudaMalloc(&g->d_gcoord, sizeof(int) * (gcoord.size() > 0 ? gcoord.size() : 3)) == cudaSuccess &&
            cudaMalloc(&g->d_status, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&g->red_partial, sizeof(double) * 5 * (size_t)(g->red_blocks > 0 ? g->red_blocks : 1)) ==
                cudaSuccess &&
            cudaMalloc(&g->red_out, sizeof(double) * 5) == cudaSuccess &&
            cudaMallocHost(&g->host_out, sizeof(double) * 5) == cudaSuccess;
  if (!ok) {
    set_error("device allocation of grid tables failed: %s", cudaGetErrorString(cudaGetLastError()));
    free_all(g);
    return CCZ4_ERR_NOMEM;
  }
  cudaMemcpy(g->d_ijk, d->ijk, sizeof(int) * 3 * (size_t)d->n_patches, cudaMemcpyHostToDevice);
  cudaMemcpy(g->d_owner, owner.data(), sizeof(int) * (size_t)slots, cudaMemcpyHostToDevice);
  if (!gcoord.empty())
    cudaMemcpy(g->d_gcoord, gcoord.data(), sizeof(int) * gcoord.size(), cudaMemcpyHostToDevice);
  cudaMemset(g->d_status, 0, sizeof(unsigned));
  if (mesh) {
    ok = upload_table(&g->d_src, mesh->src.data(), mesh->src.size()) &&
         upload_table(&g->d_interp, mesh->interp.data(), mesh->interp.size()) &&
         upload_table(&g->d_ibeg, mesh->ibeg.data(), mesh->ibeg.size()) &&
         upload_table(&g->d_xjob, mesh->xjob.data(), mesh->xjob.size()) &&
         upload_table(&g->d_yjob, mesh->yjob.data(), mesh->yjob.size()) &&
         upload_table(&g->d_zjob, mesh->zjob.data(), mesh->zjob.size()) &&
         upload_table(&g->d_xbeg, mesh->xbeg.data(), mesh->xbeg.size()) &&
         upload_table(&g->d_ybeg, mesh->ybeg.data(), mesh->ybeg.size()) &&
         upload_table(&g->d_plev, mesh->level.data(), mesh->level.size()) &&
         upload_table(&g->d_leaf, mesh->leaf.data(), mesh->leaf.size());
    for (int l = 1; l < mesh->n_levels && ok; ++l) {
      g->n_rpar[l] = (int)mesh->rpar[l].size();
      ok = upload_table(&g->d_rpar[l], mesh->rpar[l].data(), mesh->rpar[l].size()) &&
           upload_table(&g->d_rkid[l], mesh->rkid[l].data(), mesh->rkid[l].size());
    }
    if (!ok) {
      set_error("device allocation of the mesh tables failed: %s", cudaGetErrorString(cudaGetLastError()));
      free_all(g);
      return CCZ4_ERR_NOMEM;
    }
  }
  prepare_fill_halos(v.p);
  if (v.p == 9) prepare_fused();
  if (mesh) prepare_shaped_mesh();
  else prepare_shaped_uniform();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_error("grid set-up failed: %s", cudaGetErrorString(e));
    free_all(g);
    return CCZ4_ERR_CUDA;
  }
  v.ijk = g->d_ijk;
  v.owner = g->d_owner;
  v.gcoord = g->d_gcoord;
  v.status = g->d_status;
  v.src = g->d_src;
  v.interp = g->d_interp;
  v.ibeg = g->d_ibeg;
  v.xjob = g->d_xjob;
  v.yjob = g->d_yjob;
  v.zjob = g->d_zjob;
  v.xbeg = g->d_xbeg;
  v.ybeg = g->d_ybeg;
  v.plev = g->d_plev;
  v.leaf = g->d_leaf;
  if (v.n_ghost > 0) {
    // the static geometry of the Sommerfeld ghost cells, once
    if (cudaMalloc(&g->d_ghost_geo, sizeof(GhostGeo) * (size_t)v.n_ghost) != cudaSuccess) {
      set_error("device allocation of the ghost-cell geometry failed: %s", cudaGetErrorString(cudaGetLastError()));
      free_all(g);
      return CCZ4_ERR_NOMEM;
    }
    v.ghost_geo = g->d_ghost_geo;
    cudaError_t eg = launch_ghost_setup(v, g->d_ghost_geo, 0);
    if (eg == cudaSuccess) eg = cudaDeviceSynchronize();
    if (eg != cudaSuccess) {
      set_error("ghost-cell geometry set-up failed: %s", cudaGetErrorString(eg));
      free_all(g);
      return CCZ4_ERR_CUDA;
    }
  }
  *out = g;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_free_patches(ccz4_grid *g) {
  if (!g) return CCZ4_OK;
  cudaDeviceSynchronize();
  free_all(g);
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_grid_info(const ccz4_grid *g, long long *n_points, long long *n_ghost,
                                      long long *field_stride) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (n_points) *n_points = g->v.n_points;
  if (n_ghost) *n_ghost = g->v.n_ghost;
  if (field_stride) *field_stride = g->v.S;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_field_ptr(ccz4_grid *g, int buf, double **dev, long long *n_doubles) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (buf < 0 || buf > CCZ4_BUF_MIX || !g->buf[buf]) {
    set_error("buffer %d does not exist on this grid", buf);
    return CCZ4_ERR_INVALID;
  }
  if (dev) *dev = g->buf[buf];
  if (n_doubles) *n_doubles = g->buf_len[buf];
  return CCZ4_OK;
}

// Rows of doubles between a device buffer and host memory that the device
// can address (pinned, mapped): one thread per element, a warp per 32
// consecutive elements of a row, so both sides are read and written in
// full lines. Faster than a copy engine over the CPU-GPU link of a
// Grace-Blackwell node.
__global__ void __launch_bounds__(256) strided_copy_kernel(double *__restrict__ dst, long long dst_stride,
                                                            const double *__restrict__ src, long long src_stride,
                                                            long long row_len, int rows) {
  const long long total = row_len * rows;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long r = k / row_len, c = k - r * row_len;
    dst[r * dst_stride + c] = src[r * src_stride + c];
  }
}

// The device address of host memory that the device can access directly
// (pinned and mapped), or NULL.
static void *mapped_host(const void *h) {
  if (!h) return nullptr;
  const char *mode = getenv("CCZ4_HOST_COPY");
  if (mode && strcmp(mode, "dma") == 0) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA allocation: clear the error
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// rows x row_len doubles from src (stride src_stride) to dst (stride
// dst_stride), one side on the host: by the copy kernel when that side is
// mapped pinned memory, else by the copy engine.
static cudaError_t copy_rows(double *dst, long long dst_stride, const double *src, long long src_stride,
                             long long row_len, int rows, bool to_device, cudaStream_t s) {
  if (row_len <= 0 || rows <= 0) return cudaSuccess;
  void *mh = mapped_host(to_device ? (const void *)src : (const void *)dst);
  if (mh) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks_needed = (row_len * rows + 255) / 256;
    const long long blocks = blocks_needed < 8LL * sms ? blocks_needed : 8LL * sms;
    if (to_device)
      strided_copy_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, dst_stride, (const double *)mh, src_stride, row_len,
                                                            rows);
    else
      strided_copy_kernel<<<(unsigned)blocks, 256, 0, s>>>((double *)mh, dst_stride, src, src_stride, row_len, rows);
    return cudaGetLastError();
  }
  return cudaMemcpy2DAsync(dst, sizeof(double) * dst_stride, src, sizeof(double) * src_stride,
                           sizeof(double) * row_len, rows, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                           s);
}

static ccz4_status copy_state(ccz4_grid *g, int buf, double *U, double *G, bool to_device, cudaStream_t s) {
  const GridView &v = g->v;
  double *d = g->buf[buf];
  if (v.n_points > 0) {
    if (to_device)
      CUDA_TRY(copy_rows(d, v.S, U, v.n_points, v.n_points, NV, true, s));
    else
      CUDA_TRY(copy_rows(U, v.n_points, d, v.S, v.n_points, NV, false, s));
  }
  if (v.n_ghost > 0 && G) {
    if (to_device)
      CUDA_TRY(copy_rows(d + v.n_points, v.S, G, v.n_ghost, v.n_ghost, NV, true, s));
    else
      CUDA_TRY(copy_rows(G, v.n_ghost, d + v.n_points, v.S, v.n_ghost, NV, false, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_upload(ccz4_grid *g, int buf, const double *U, const double *G, void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (!state_buffer(buf) || !g->buf[buf] || (!U && g->v.n_points > 0)) {
    set_error("upload: invalid buffer %d or NULL host array", buf);
    return CCZ4_ERR_INVALID;
  }
  if (g->v.n_ghost > 0 && !G) {
    set_error("upload: this grid has %lld Sommerfeld ghost cells; G must be given", g->v.n_ghost);
    return CCZ4_ERR_INVALID;
  }
  return copy_state(g, buf, const_cast<double *>(U), const_cast<double *>(G), true, (cudaStream_t)stream);
}

extern "C" ccz4_status ccz4_download(ccz4_grid *g, int buf, double *U, double *G, void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (buf == CCZ4_BUF_TILE || buf == CCZ4_BUF_MIX) {
    if (!U) {
      set_error("download: NULL host array");
      return CCZ4_ERR_INVALID;
    }
    CUDA_TRY(cudaMemcpyAsync(U, g->buf[buf], sizeof(double) * (size_t)g->buf_len[buf], cudaMemcpyDeviceToHost,
                             (cudaStream_t)stream));
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return CCZ4_OK;
  }
  if (!state_buffer(buf) || !g->buf[buf] || (!U && g->v.n_points > 0)) {
    set_error("download: invalid buffer %d or NULL host array", buf);
    return CCZ4_ERR_INVALID;
  }
  return copy_state(g, buf, U, G, false, (cudaStream_t)stream);
}

extern "C" ccz4_status ccz4_fill_halos(ccz4_grid *g, int buf, void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (!state_buffer(buf) || !g->buf[buf]) {
    set_error("fill_halos: buffer %d is not a state buffer of this grid", buf);
    return CCZ4_ERR_INVALID;
  }
  CUDA_TRY(launch_fill_halos(g->v, g->buf[buf], g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], (cudaStream_t)stream));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_fill_halos_for(ccz4_grid *g, int buf, const ccz4_params *P, void *stream) {
  if (check_grid(g) || check_params(P)) return CCZ4_ERR_INVALID;
  if (!state_buffer(buf) || !g->buf[buf]) {
    set_error("fill_halos_for: buffer %d is not a state buffer of this grid", buf);
    return CCZ4_ERR_INVALID;
  }
  CUDA_TRY(launch_fill_halos(g->v, g->buf[buf], g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], (cudaStream_t)stream,
                             P->precision == CCZ4_PREC_MIXED));
  return CCZ4_OK;
}

static const double *ini_ptr(ccz4_grid *g) {
  return g->buf[CCZ4_BUF_INI] ? g->buf[CCZ4_BUF_INI] : g->buf[CCZ4_BUF_U];
}

extern "C" ccz4_status ccz4_rhs(ccz4_grid *g, const ccz4_params *P, int in_buf, int out_buf, void *stream) {
  if (check_grid(g) || check_params(P)) return CCZ4_ERR_INVALID;
  if (!state_buffer(in_buf) || !state_buffer(out_buf) || in_buf == out_buf || !g->buf[in_buf] ||
      !g->buf[out_buf] || out_buf == CCZ4_BUF_INI) {
    set_error("rhs: invalid buffers in=%d out=%d", in_buf, out_buf);
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(launch_fill_halos(g->v, g->buf[in_buf], g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], s,
                             P->precision == CCZ4_PREC_MIXED));
  CUDA_TRY(launch_rhs(g->v, *P, g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], g->buf[in_buf], ini_ptr(g), g->buf[out_buf], s));
  return CCZ4_OK;
}

static const int kStageIn[4] = {CCZ4_BUF_U, CCZ4_BUF_Y0, CCZ4_BUF_Y1, CCZ4_BUF_Y0};
static const int kStageOut[4] = {CCZ4_BUF_Y0, CCZ4_BUF_Y1, CCZ4_BUF_Y0, CCZ4_BUF_U};

// Restriction of every refined level onto the one below, finest first.
static ccz4_status restrict_levels(ccz4_grid *g, double *U, cudaStream_t s) {
  for (int l = g->v.n_levels - 1; l >= 1; --l)
    CUDA_TRY(launch_restrict(g->v, g->d_rpar[l], g->d_rkid[l], g->n_rpar[l], U, s));
  return CCZ4_OK;
}

// One RK4 stage from the halo'd tiles; stage 3 ends the step (enforcement
// in the stage kernel, then the restriction on a mesh).
static ccz4_status stage_kernel(ccz4_grid *g, const ccz4_params *P, int stage, double dt, cudaStream_t s) {
  double *in = g->buf[kStageIn[stage]];
  CUDA_TRY(launch_rk_stage(g->v, *P, stage, dt, g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], in, ini_ptr(g), g->buf[CCZ4_BUF_U],
                           g->buf[CCZ4_BUF_ACC], g->buf[kStageOut[stage]], s));
  if (stage == 3 && g->v.n_levels > 1) return restrict_levels(g, g->buf[kStageOut[stage]], s);
  return CCZ4_OK;
}

// One RK4 stage of a step: the halo fill and the stage kernel as two
// launches, or (CCZ4_LAUNCH_FUSED) both in one cooperative launch; the
// restriction after stage 3 stays a launch of its own.
static ccz4_status step_stage(ccz4_grid *g, const ccz4_params *P, int stage, double dt, cudaStream_t s) {
  if (!g->fused) {
    CUDA_TRY(launch_fill_halos(g->v, g->buf[kStageIn[stage]], g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], s,
                               P->precision == CCZ4_PREC_MIXED));
    return stage_kernel(g, P, stage, dt, s);
  }
  CUDA_TRY(launch_fused_stage(g->v, *P, stage, dt, g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX],
                              g->buf[kStageIn[stage]], ini_ptr(g), g->buf[CCZ4_BUF_U], g->buf[CCZ4_BUF_ACC],
                              g->buf[kStageOut[stage]], s));
  if (stage == 3 && g->v.n_levels > 1) return restrict_levels(g, g->buf[kStageOut[stage]], s);
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_set_launch(ccz4_grid *g, int mode) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (mode != CCZ4_LAUNCH_FLAT && mode != CCZ4_LAUNCH_QUEUE && mode != CCZ4_LAUNCH_FUSED) {
    set_error("set_launch: unknown launch mode %d", mode);
    return CCZ4_ERR_INVALID;
  }
  if (mode == CCZ4_LAUNCH_FUSED && g->v.p != 9) {
    set_error("set_launch: the fused stage launch is compiled for 9^3 patches (this grid has %d^3)", g->v.p);
    return CCZ4_ERR_INVALID;
  }
  if (mode == CCZ4_LAUNCH_QUEUE && !g->d_queue) {
    if (cudaMalloc(&g->d_queue, sizeof(unsigned long long)) != cudaSuccess) {
      set_error("set_launch: allocation of the work counter failed: %s", cudaGetErrorString(cudaGetLastError()));
      return CCZ4_ERR_NOMEM;
    }
  }
  unsigned long long *q = mode == CCZ4_LAUNCH_QUEUE ? g->d_queue : nullptr;
  const int fused = mode == CCZ4_LAUNCH_FUSED;
  if ((q != g->v.queue || fused != g->fused) && g->step_exec) {
    cudaGraphExecDestroy(g->step_exec);  // the captured step used the other launch
    g->step_exec = nullptr;
  }
  g->v.queue = q;
  g->fused = fused;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_set_tuning(ccz4_grid *g, int stage_shape, int fill_shape) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (stage_shape < 0 || stage_shape > 3 || fill_shape < 0 || fill_shape > 3) {
    set_error("set_tuning: stage shape must be 0..3 and fill shape 0..3 (got %d, %d)", stage_shape, fill_shape);
    return CCZ4_ERR_INVALID;
  }
  if ((stage_shape != g->v.stage_shape || fill_shape != g->v.fill_shape) && g->step_exec) {
    cudaGraphExecDestroy(g->step_exec);  // the captured step used the other shapes
    g->step_exec = nullptr;
  }
  g->v.stage_shape = stage_shape;
  g->v.fill_shape = fill_shape;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_restrict(ccz4_grid *g, int buf, void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (!state_buffer(buf) || !g->buf[buf]) {
    set_error("restrict: buffer %d is not a state buffer of this grid", buf);
    return CCZ4_ERR_INVALID;
  }
  return restrict_levels(g, g->buf[buf], (cudaStream_t)stream);
}

extern "C" ccz4_status ccz4_stage_buffers(int stage, int *in_buf, int *out_buf) {
  if (stage < 0 || stage > 3) {
    set_error("stage must be 0..3 (got %d)", stage);
    return CCZ4_ERR_INVALID;
  }
  if (in_buf) *in_buf = kStageIn[stage];
  if (out_buf) *out_buf = kStageOut[stage];
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_rk_stage(ccz4_grid *g, const ccz4_params *P, int stage, double dt, void *stream) {
  if (check_grid(g) || check_params(P)) return CCZ4_ERR_INVALID;
  if (stage < 0 || stage > 3 || !(dt == dt)) {
    set_error("rk_stage: stage must be 0..3 (got %d) and dt finite", stage);
    return CCZ4_ERR_INVALID;
  }
  return stage_kernel(g, P, stage, dt, (cudaStream_t)stream);
}

extern "C" ccz4_status ccz4_step(ccz4_grid *g, const ccz4_params *P, double dt, int n_steps, void *stream) {
  if (check_grid(g) || check_params(P)) return CCZ4_ERR_INVALID;
  if (n_steps < 0 || !(dt == dt)) {
    set_error("step: n_steps must be >= 0 and dt finite");
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  for (int n = 0; n < n_steps; ++n)
    for (int st = 0; st < 4; ++st) {
      ccz4_status r = step_stage(g, P, st, dt, s);
      if (r != CCZ4_OK) return r;
    }
  return CCZ4_OK;
}

// Captures one RK4 step (four halo fills and four stage launches) into a
// CUDA graph on a private stream; kernel arguments, parameters and dt are
// baked into the graph.
static ccz4_status capture_step(ccz4_grid *g, const ccz4_params *P, double dt) {
  if (g->step_exec) {
    cudaGraphExecDestroy(g->step_exec);
    g->step_exec = nullptr;
  }
  if (!g->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
  ccz4_status st = CCZ4_OK;
  for (int s = 0; s < 4 && st == CCZ4_OK; ++s) st = step_stage(g, P, s, dt, g->cap_stream);
  cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
  if (st != CCZ4_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) {
    set_error("cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&g->step_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->step_exec = nullptr;
    set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  g->step_P = *P;
  g->step_dt = dt;
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_step_graph(ccz4_grid *g, const ccz4_params *P, double dt, int n_steps, void *stream) {
  if (check_grid(g) || check_params(P)) return CCZ4_ERR_INVALID;
  if (n_steps < 0 || !(dt == dt)) {
    set_error("step_graph: n_steps must be >= 0 and dt finite");
    return CCZ4_ERR_INVALID;
  }
  if (n_steps == 0) return CCZ4_OK;
  if (!g->step_exec || memcmp(&g->step_P, P, sizeof(ccz4_params)) != 0 || g->step_dt != dt) {
    // the graph's first kernel must not start before earlier work on `stream`
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    ccz4_status st = capture_step(g, P, dt);
    if (st != CCZ4_OK) return st;
  }
  for (int n = 0; n < n_steps; ++n) CUDA_TRY(cudaGraphLaunch(g->step_exec, (cudaStream_t)stream));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_evolve_host(ccz4_grid *g, const ccz4_params *P, double dt, int n_steps,
                                        const double *U_in, const double *G_in, double *U_out, double *G_out,
                                        void *stream) {
  ccz4_status st = ccz4_upload(g, CCZ4_BUF_U, U_in, G_in, stream);
  if (st != CCZ4_OK) return st;
  st = ccz4_step(g, P, dt, n_steps, stream);
  if (st != CCZ4_OK) return st;
  return ccz4_download(g, CCZ4_BUF_U, U_out, G_out, stream);
}

extern "C" ccz4_status ccz4_enforce(ccz4_grid *g, int buf, void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (!state_buffer(buf) || !g->buf[buf]) {
    set_error("enforce: buffer %d is not a state buffer of this grid", buf);
    return CCZ4_ERR_INVALID;
  }
  CUDA_TRY(launch_enforce(g->v, g->buf[buf], (cudaStream_t)stream));
  return CCZ4_OK;
}

namespace {
// One thread per queried lattice point: its index within a field of a
// state buffer, resolved as the halo fill resolves tile points (locate);
// points beyond the ghost shell set the bounds bit of v.status.
__global__ void __launch_bounds__(256) point_index_kernel(ccz4::GridView v, int n, const int *__restrict__ xyz,
                                                          long long *__restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  out[q] = ccz4::locate(v, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2]);
}
}  // namespace

extern "C" ccz4_status ccz4_point_index(ccz4_grid *g, int n, const int *xyz, long long *index, void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (n < 0 || n > (1 << 20) || (n > 0 && (!xyz || !index))) {
    set_error("point_index: need 0 <= n <= 2^20 points and host arrays xyz and index");
    return CCZ4_ERR_INVALID;
  }
  if (g->v.n_levels > 1 || g->v.src) {
    set_error("point_index: lattice indices address a single uniform level, not a refined mesh");
    return CCZ4_ERR_INVALID;
  }
  if (n == 0) return CCZ4_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int *d_xyz = nullptr;
  long long *d_idx = nullptr;
  unsigned *d_st = nullptr;
  if (cudaMalloc(&d_xyz, sizeof(int) * 3 * (size_t)n) != cudaSuccess ||
      cudaMalloc(&d_idx, sizeof(long long) * (size_t)n) != cudaSuccess ||
      cudaMalloc(&d_st, sizeof(unsigned)) != cudaSuccess) {
    set_error("point_index: device allocation failed: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(d_xyz);
    cudaFree(d_idx);
    cudaFree(d_st);
    return CCZ4_ERR_NOMEM;
  }
  ccz4::GridView v = g->v;
  v.status = d_st;  // this call's own bounds status
  unsigned status = 0;
  cudaError_t e = cudaMemsetAsync(d_st, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_xyz, xyz, sizeof(int) * 3 * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    point_index_kernel<<<(n + 255) / 256, 256, 0, s>>>(v, n, d_xyz, d_idx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(index, d_idx, sizeof(long long) * (size_t)n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_st, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_xyz);
  cudaFree(d_idx);
  cudaFree(d_st);
  if (e != cudaSuccess) {
    set_error("point_index: %s", cudaGetErrorString(e));
    return CCZ4_ERR_CUDA;
  }
  if (status & STATUS_BOUNDS) {
    long long bad = 0;
    for (int q = 0; q < n; ++q) bad += index[q] < 0;
    set_error("point_index: %lld of %d points lie outside the grid and its ghost shell", bad, n);
    return CCZ4_ERR_BOUNDS;
  }
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_psi4(ccz4_grid *g, int in_buf, int out_buf, const double centre[3], void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (!state_buffer(in_buf) || !state_buffer(out_buf) || in_buf == out_buf || !g->buf[in_buf] ||
      !g->buf[out_buf] || !centre || !(centre[0] == centre[0] && centre[1] == centre[1] && centre[2] == centre[2])) {
    set_error("psi4: need two different state buffers (in=%d out=%d) and a finite centre", in_buf, out_buf);
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(launch_fill_halos(g->v, g->buf[in_buf], g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], s));
  CUDA_TRY(launch_psi4(g->v, g->buf[CCZ4_BUF_TILE], centre, g->buf[out_buf], s));
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_constraints(ccz4_grid *g, int buf, double out[5], double *dev_H, double *dev_M,
                                        void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (!state_buffer(buf) || !g->buf[buf] || !out) {
    set_error("constraints: invalid buffer %d or NULL out", buf);
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(launch_fill_halos(g->v, g->buf[buf], g->buf[CCZ4_BUF_TILE], g->buf[CCZ4_BUF_MIX], s));
  CUDA_TRY(launch_constraints(g->v, g->buf[CCZ4_BUF_TILE], dev_H, dev_M, g->red_partial, g->red_blocks,
                              g->red_out, s));
  CUDA_TRY(cudaMemcpyAsync(g->host_out, g->red_out, sizeof(double) * 5, cudaMemcpyDeviceToHost, s));
  unsigned status = 0;
  CUDA_TRY(cudaMemcpyAsync(&status, g->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  memcpy(out, g->host_out, sizeof(double) * 5);
  if (status & STATUS_BOUNDS) {
    set_error("a kernel met a point outside the grid (device status %u)", status);
    return CCZ4_ERR_BOUNDS;
  }
  if (out[4] > 0.0) {
    set_error("%.0f points have non-finite constraint values", out[4]);
    return CCZ4_ERR_NONFINITE;
  }
  return CCZ4_OK;
}

extern "C" ccz4_status ccz4_constraints_excluding(ccz4_grid *g, const double *dev_H, const double *dev_M,
                                                  int n_centres, const double *centres, double radius,
                                                  double out[5], void *stream) {
  if (check_grid(g)) return CCZ4_ERR_INVALID;
  if (!dev_H || !dev_M || !out || n_centres < 0 || n_centres > CCZ4_MAX_EXCLUDED || (n_centres > 0 && !centres) ||
      !(radius >= 0.0)) {
    set_error("constraints_excluding: dev_H, dev_M and out must be given, 0 <= n_centres <= %d, radius >= 0",
              CCZ4_MAX_EXCLUDED);
    return CCZ4_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(launch_constraints_excluded(g->v, dev_H, dev_M, n_centres, centres, radius, g->red_partial,
                                       g->red_blocks, g->red_out, s));
  CUDA_TRY(cudaMemcpyAsync(g->host_out, g->red_out, sizeof(double) * 5, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  memcpy(out, g->host_out, sizeof(double) * 5);
  return CCZ4_OK;
}

extern "C" const char *ccz4_last_error(void) { return g_err; }
