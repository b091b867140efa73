// aux.cu — kernels off the hot path: L2 projection of initial conditions, the initial CFL rate
// reduction, conversion between the canonical FP64 layout and the FP32-form storage, and
// deterministic mass sums.
#include <math.h>

#include "dg_internal.h"

namespace dgk {

__constant__ double c_gx[9][8];
__constant__ double c_gw[9][8];

template <int N>
static void put_rule(double (&gx)[9][8], double (&gw)[9][8]) {
  for (int i = 0; i < N; ++i) {
    gx[N][i] = GaussRule<N>::x(i);
    gw[N][i] = GaussRule<N>::w(i);
  }
}

cudaError_t aux_init_tables() {
  double gx[9][8] = {}, gw[9][8] = {};
  put_rule<1>(gx, gw);
  put_rule<2>(gx, gw);
  put_rule<3>(gx, gw);
  put_rule<4>(gx, gw);
  put_rule<5>(gx, gw);
  put_rule<6>(gx, gw);
  put_rule<7>(gx, gw);
  put_rule<8>(gx, gw);
  cudaError_t e = cudaMemcpyToSymbol(c_gx, gx, sizeof(gx));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_gw, gw, sizeof(gw));
}

size_t state_bytes(const AuxGeom& g) {
  if (g.prec == PREC_F64) return sizeof(double) * (size_t)g.nv * g.nm * g.ncell;
  return F32Layout{g.ncell, g.nv, g.nm}.bytes();
}

// P_l(x) by the three-term recurrence.
__device__ inline double leg(int l, double x) {
  double pm = 1.0, p = x;
  if (l == 0) return 1.0;
  for (int j = 1; j < l; ++j) {
    double pn = ((2.0 * j + 1.0) * x * p - j * pm) / (j + 1.0);
    pm = p;
    p = pn;
  }
  return p;
}

struct IcParams {
  int kind, nprm;
  double p[20];
};

// Conservative state of an analytic initial condition at (x, y).
__device__ void ic_eval(const AuxGeom& g, const IcParams& ic, double x, double y, double* U) {
  const double gam = g.gamma;
  switch (ic.kind) {
    case 0: {  // a + b sin(w (x [+ y]) + phi)
      const double s = g.dim == 2 ? x + y : x;
      U[0] = ic.p[0] + ic.p[1] * sin(ic.p[2] * s + ic.p[3]);
      return;
    }
    case 1: {  // 1D Riemann: left/right primitive states, split at p[6]
      const double* W = x < ic.p[6] ? ic.p : ic.p + 3;
      U[0] = W[0];
      U[1] = W[0] * W[1];
      U[2] = W[2] / (gam - 1.0) + 0.5 * W[0] * W[1] * W[1];
      return;
    }
    case 2: {  // entropy wave rho = r0 + A sin(w x), u = u0, p = p0
      const double rho = ic.p[0] + ic.p[1] * sin(ic.p[2] * x);
      U[0] = rho;
      U[1] = rho * ic.p[3];
      U[2] = ic.p[4] / (gam - 1.0) + 0.5 * rho * ic.p[3] * ic.p[3];
      return;
    }
    case 3: {  // four quadrants Q1 (x>xs,y>ys), Q2 (x<xs,y>ys), Q3 (x<xs,y<ys), Q4 (x>xs,y<ys)
      const bool right = x > ic.p[16], upper = y > ic.p[17];
      const int qd = right ? (upper ? 0 : 3) : (upper ? 1 : 2);
      const double* W = ic.p + 4 * qd;
      U[0] = W[0];
      U[1] = W[0] * W[1];
      U[2] = W[0] * W[2];
      U[3] = W[3] / (gam - 1.0) + 0.5 * W[0] * (W[1] * W[1] + W[2] * W[2]);
      return;
    }
    case 4: {  // isentropic vortex of Example 3.4(a), centre (x0 + t, y0), nearest periodic image
      const double Lx = g.hx * g.nx, Ly = g.hy * g.ny;
      double dx = x - ic.p[3] - ic.p[0], dy = y - ic.p[1];
      dx -= Lx * floor(dx / Lx + 0.5);
      dy -= Ly * floor(dy / Ly + 0.5);
      const double bet = ic.p[2];
      const double e = exp(1.0 - (dx * dx + dy * dy));
      const double rho = pow(1.0 - (gam - 1.0) / (16.0 * gam * M_PI * M_PI) * bet * bet * e * e, 1.0 / (gam - 1.0));
      const double uu = 1.0 - bet * e * dy / (2.0 * M_PI);
      const double vv = bet * e * dx / (2.0 * M_PI);
      const double pp = pow(rho, gam);
      U[0] = rho;
      U[1] = rho * uu;
      U[2] = rho * vv;
      U[3] = pp / (gam - 1.0) + 0.5 * rho * (uu * uu + vv * vv);
      return;
    }
  }
}

__global__ void project_kernel(const AuxGeom g, const IcParams ic, int nq, double* out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int i = (int)(c % g.nx), j = (int)(c / g.nx);
  const double xc = g.x0 + (i + 0.5) * g.hx, yc = g.y0 + (j + 0.5) * g.hy;
  double acc[4][16];
  for (int v = 0; v < g.nv; ++v)
    for (int m = 0; m < g.nm; ++m) acc[v][m] = 0.0;
  const int nb = g.dim == 2 ? nq : 1;
  for (int a = 0; a < nq; ++a)
    for (int b = 0; b < nb; ++b) {
      const double xi = c_gx[nq][a], eta = g.dim == 2 ? c_gx[nq][b] : 0.0;
      const double w = c_gw[nq][a] * (g.dim == 2 ? c_gw[nq][b] : 1.0);
      double U[4];
      ic_eval(g, ic, xc + 0.5 * g.hx * xi, yc + 0.5 * g.hy * eta, U);
      for (int m = 0; m < g.nm; ++m) {
        const double phi = leg(g.mp[m], xi) * (g.dim == 2 ? leg(g.mq[m], eta) : 1.0);
        for (int v = 0; v < g.nv; ++v) acc[v][m] += w * U[v] * phi;
      }
    }
  for (int m = 0; m < g.nm; ++m) {
    // 1 / int P_p^2 P_q^2 on the reference cell = (2p+1)(2q+1)/4 (1D: (2l+1)/2)
    const double inv = g.dim == 2 ? 0.25 * (2 * g.mp[m] + 1) * (2 * g.mq[m] + 1) : 0.5 * (2 * g.mp[m] + 1);
    for (int v = 0; v < g.nv; ++v) out[((long long)v * g.nm + m) * g.ncell + c] = acc[v][m] * inv;
  }
}

cudaError_t launch_project(const AuxGeom& g, int ic, const double* prm, int nprm, int nq,
                           double* canon_out, cudaStream_t s) {
  IcParams p{};
  p.kind = ic;
  p.nprm = nprm;
  for (int i = 0; i < nprm && i < 20; ++i) p.p[i] = prm[i];
  const unsigned blocks = (unsigned)((g.ncell + 127) / 128);
  project_kernel<<<blocks, 128, 0, s>>>(g, p, nq, canon_out);
  return cudaGetLastError();
}

// Cell average of variable v from either storage form.
__device__ inline double avg_of(const AuxGeom& g, const void* st, int v, long long c) {
  if (g.prec == PREC_F64) return ((const double*)st)[((long long)v * g.nm) * g.ncell + c];
  const F32Layout L{g.ncell, g.nv, g.nm};
  const float* b = (const float*)st;
  return (double)b[L.word(v, 0, c)] + (double)b[L.word(v, g.nm, c)];
}

// Coefficient (v, m) of cell c from either storage form.
__device__ inline double coef_of(const AuxGeom& g, const void* st, int v, int m, long long c) {
  if (m == 0) return avg_of(g, st, v, c);
  if (g.prec == PREC_F64) return ((const double*)st)[((long long)v * g.nm + m) * g.ncell + c];
  return (double)((const float*)st)[F32Layout{g.ncell, g.nv, g.nm}.word(v, m, c)];
}

// CFL rate of one state: beta^x / hx (+ beta^y / hy).
__device__ inline double state_rate(const AuxGeom& g, const double* ub, bool& phys) {
  double bx, by, invH;
  if (g.eq == EQ_EULER) {
    if (g.dim == 1) avg_params<EQ_EULER, 1>(ub, g.gamma, g.gamma - 1.0, g.ax, g.ay, bx, by, invH, phys);
    else avg_params<EQ_EULER, 2>(ub, g.gamma, g.gamma - 1.0, g.ax, g.ay, bx, by, invH, phys);
  } else if (g.eq == EQ_BURG) {
    avg_params<EQ_BURG, 2>(ub, g.gamma, g.gamma - 1.0, g.ax, g.ay, bx, by, invH, phys);
  } else {
    avg_params<EQ_ADV, 2>(ub, g.gamma, g.gamma - 1.0, g.ax, g.ay, bx, by, invH, phys);
  }
  return bx / g.hx + (g.dim == 2 ? by / g.hy : 0.0);
}

// Max CFL rate over the cells' averages; with the positivity limiter also over its points (the
// k+1 Gauss points per direction of the volume and the edges, 1D: Gauss points and both ends; for
// k = 3 also the Gauss-Lobatto mid-lines xi = 0 and eta = 0 crossed with the Gauss nodes, 1D: 0).
__global__ void rate_kernel(const AuxGeom g, const void* st, DevScalars* sc, int slot) {
  __shared__ double red[32];
  double r = 0.0;
  bool ok = true;
  const int nq = g.k + 1;
  const int mid = (g.k >= 2 && nq % 2 == 0) ? 1 : 0;
  const int npt = !g.pp ? 0 : (g.dim == 1 ? nq + 2 + mid : nq * nq + 4 * nq + 2 * nq * mid);
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double ub[4];
    for (int v = 0; v < g.nv; ++v) ub[v] = avg_of(g, st, v, c);
    bool phys;
    double rc = state_rate(g, ub, phys);
    r = (rc > r || rc != rc) ? rc : r;
    ok = ok && phys;
    for (int i = 0; i < npt; ++i) {
      double xi, eta = 0.0;
      if (g.dim == 1) {
        xi = i < nq ? c_gx[nq][i] : (i == nq ? -1.0 : (i == nq + 1 ? 1.0 : 0.0));
      } else if (i < nq * nq) {
        xi = c_gx[nq][i / nq];
        eta = c_gx[nq][i % nq];
      } else if (i >= nq * nq + 4 * nq) {
        const int j = i - nq * nq - 4 * nq, gq = j >> 1;
        xi = (j & 1) ? c_gx[nq][gq] : 0.0;
        eta = (j & 1) ? 0.0 : c_gx[nq][gq];
      } else {
        const int e = (i - nq * nq) & 3, gq = (i - nq * nq) >> 2;
        xi = e == 0 ? -1.0 : (e == 1 ? 1.0 : c_gx[nq][gq]);
        eta = e == 2 ? -1.0 : (e == 3 ? 1.0 : c_gx[nq][gq]);
      }
      double w[4] = {0.0, 0.0, 0.0, 0.0};
      for (int m = 0; m < g.nm; ++m) {
        const double phi = leg(g.mp[m], xi) * (g.dim == 2 ? leg(g.mq[m], eta) : 1.0);
        for (int v = 0; v < g.nv; ++v) w[v] += phi * coef_of(g, st, v, m, c);
      }
      bool pphys;
      const double rp = state_rate(g, w, pphys);
      r = (rp > r || rp != rp) ? rp : r;
    }
  }
  r = warp_max(r);
  const unsigned bad = __ballot_sync(0xffffffffu, !ok);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = (red[w] > m || red[w] != red[w]) ? red[w] : m;
    atomic_max_nonneg(&sc->rate_bits[slot], m);
  }
  if (bad && (threadIdx.x & 31) == 0) atomicOr(&sc->err, ERRB_NONPHYS);
}

cudaError_t launch_rate(const AuxGeom& g, const void* state, DevScalars* sc, int slot, cudaStream_t s) {
  unsigned blocks = (unsigned)((g.ncell + 255) / 256);
  if (blocks > 1216) blocks = 1216;
  rate_kernel<<<blocks, 256, 0, s>>>(g, state, sc, slot);
  return cudaGetLastError();
}

__global__ void to_storage_kernel(const AuxGeom g, const double* canon, void* st) {
  const long long total = (long long)g.nv * g.nm * g.ncell;
  const F32Layout L{g.ncell, g.nv, g.nm};
  float* b = (float*)st;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e % g.ncell, vm = e / g.ncell;
    const int v = (int)(vm / g.nm), m = (int)(vm % g.nm);
    const double x = canon[e];
    if (m == 0) {
      const float hi = (float)x;
      b[L.word(v, 0, c)] = hi;
      b[L.word(v, g.nm, c)] = (float)(x - (double)hi);
    } else {
      b[L.word(v, m, c)] = (float)x;
    }
  }
}

__global__ void from_storage_kernel(const AuxGeom g, const void* st, double* canon) {
  const long long total = (long long)g.nv * g.nm * g.ncell;
  const F32Layout L{g.ncell, g.nv, g.nm};
  const float* b = (const float*)st;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e % g.ncell, vm = e / g.ncell;
    const int v = (int)(vm / g.nm), m = (int)(vm % g.nm);
    if (m == 0) {
      canon[e] = (double)b[L.word(v, 0, c)] + (double)b[L.word(v, g.nm, c)];
    } else {
      canon[e] = (double)b[L.word(v, m, c)];
    }
  }
}

int hybrid_lmax(const AuxGeom& g) { return g.dim == 1 ? g.k : (g.basis == 0 ? 2 * g.k : g.k); }

// Algorithm 1, after a stage kernel that stored the DG solution: on each listed troubled cell,
// u^hyd = omega u^DG + (1 - omega) u^lim with u^lim's mode of total degree l equal to
// exp(-sigma^l dt) u^DG's, i.e. each higher mode scaled by omega + (1 - omega) exp(-sigma^l dt),
// omega = (max eta - eta) / (max eta - 1). Cell averages are untouched. The last block to finish
// clears the count and the maximum for the next stage.
__global__ void hybrid_blend_kernel(const AuxGeom g, void* st, const HybridOut h) {
  volatile HybridScalars* vs = h.sc;
  const unsigned n = vs->count;
  const double emax = __longlong_as_double((long long)vs->max_bits);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long c = h.list[i];
    if (g.prec == PREC_F64) {
      const double e = ((const double*)h.eta)[c];
      const double w = (emax - e) / (emax - 1.0);
      double* b = (double*)st;
      for (int m = 1; m < g.nm; ++m) {
        const int l = g.mp[m] + g.mq[m];
        const double f = w + (1.0 - w) * ((const double*)h.fac)[(long long)(l - 1) * g.ncell + c];
        for (int v = 0; v < g.nv; ++v) b[((long long)v * g.nm + m) * g.ncell + c] *= f;
      }
    } else {
      const float e = ((const float*)h.eta)[c];
      const float w = (float)((emax - (double)e) / (emax - 1.0));
      const F32Layout L{g.ncell, g.nv, g.nm};
      float* b = (float*)st;
      for (int m = 1; m < g.nm; ++m) {
        const int l = g.mp[m] + g.mq[m];
        const float f = w + (1.0f - w) * ((const float*)h.fac)[(long long)(l - 1) * g.ncell + c];
        for (int v = 0; v < g.nv; ++v) b[L.word(v, m, c)] *= f;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&h.sc->blocks, 1u);
    if (prev == gridDim.x - 1) {
      vs->count = 0u;
      vs->max_bits = 0ull;
      vs->blocks = 0u;
      __threadfence();
    }
  }
}

cudaError_t launch_hybrid_blend(const AuxGeom& g, void* state, const HybridOut& h, cudaStream_t s) {
  hybrid_blend_kernel<<<304, 256, 0, s>>>(g, state, h);
  return cudaGetLastError();
}

// OEDG damping (Section 2.1 as the paper restates it), after the stage kernel stored u~ and the jump
// sums: per variable v the normaliser N_v = ||u_v - avg u_v||_inf = max(max_v - avg_v, avg_v - min_v)
// over the volume Gauss points, c_v = 1 / (2 (2k-1) N_v) (0 if N_v = 0, u_v constant), and per cell
// sigma^l = max_v c_v A_v(l); the modes of total degree l >= 1 are multiplied by exp(-sigma^l dt).
__global__ void oedg_filter_kernel(const AuxGeom g, void* st, const OedgOut o, const DevScalars* sc) {
  volatile OedgScalars* vs = o.sc;
  if (!vs->active) return;                      // the stage did not run (solve finished or failed)
  const int lmax = g.dim == 1 ? g.k : (g.basis == 0 ? 2 * g.k : g.k);
  double cv[4];
  for (int v = 0; v < g.nv; ++v) {
    const double avg = vs->sum[v] / (double)g.ncell;
    const double mx = from_ordered_bits(vs->maxb[v]), mn = from_ordered_bits(~vs->nminb[v]);
    const double n = fmax(mx - avg, avg - mn);
    cv[v] = n > 0.0 ? 1.0 / (2.0 * (2 * g.k - 1) * n) : 0.0;
  }
  const double dt = ((volatile DevScalars*)sc)->dt;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double fac[7];
    for (int l = 1; l <= lmax; ++l) {
      double best = 0.0;
      for (int v = 0; v < g.nv; ++v) {
        const long long i = (long long)(v * lmax + l - 1) * g.ncell + c;
        const double a = g.prec == PREC_F64 ? ((const double*)o.A)[i] : (double)((const float*)o.A)[i];
        const double sv = cv[v] * a;
        best = (sv > best || sv != sv) ? sv : best;
      }
      fac[l] = exp(-best * dt);
    }
    if (g.prec == PREC_F64) {
      double* b = (double*)st;
      for (int m = 1; m < g.nm; ++m) {
        const double f = fac[g.mp[m] + g.mq[m]];
        for (int v = 0; v < g.nv; ++v) b[((long long)v * g.nm + m) * g.ncell + c] *= f;
      }
    } else {
      const F32Layout L{g.ncell, g.nv, g.nm};
      float* b = (float*)st;
      for (int m = 1; m < g.nm; ++m) {
        const float f = (float)fac[g.mp[m] + g.mq[m]];
        for (int v = 0; v < g.nv; ++v) b[L.word(v, m, c)] *= f;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&o.sc->blocks, 1u);
    if (prev == gridDim.x - 1) {                // every block has read the reductions: clear them
      for (int v = 0; v < 4; ++v) {
        vs->sum[v] = 0.0;
        vs->maxb[v] = 0ull;
        vs->nminb[v] = 0ull;
      }
      vs->active = 0u;
      vs->blocks = 0u;
      __threadfence();
    }
  }
}

cudaError_t launch_oedg_filter(const AuxGeom& g, void* state, const OedgOut& o, const DevScalars* sc,
                               cudaStream_t s) {
  oedg_filter_kernel<<<1216, 256, 0, s>>>(g, state, o, sc);
  return cudaGetLastError();
}

cudaError_t launch_to_storage(const AuxGeom& g, const double* canon, void* state, cudaStream_t s) {
  to_storage_kernel<<<1216, 256, 0, s>>>(g, canon, state);
  return cudaGetLastError();
}

cudaError_t launch_from_storage(const AuxGeom& g, const void* state, double* canon, cudaStream_t s) {
  from_storage_kernel<<<1216, 256, 0, s>>>(g, state, canon);
  return cudaGetLastError();
}

// Deterministic mass: MASS_BLOCKS fixed partial sums per variable, then one ordered final sum.
__global__ void mass_partial_kernel(const AuxGeom g, const void* st, double* partials) {
  __shared__ double red[256];
  for (int v = 0; v < g.nv; ++v) {
    double s = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x)
      s += avg_of(g, st, v, c);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[v * gridDim.x + blockIdx.x] = red[0];
    __syncthreads();
  }
}

__global__ void mass_final_kernel(const AuxGeom g, const double* partials, int nparts, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int v = 0; v < g.nv; ++v) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partials[v * nparts + b];
    out[v] = s * g.hx * (g.dim == 2 ? g.hy : 1.0);
  }
}

cudaError_t launch_mass(const AuxGeom& g, const void* state, double* partials, double* out, cudaStream_t s) {
  mass_partial_kernel<<<MASS_BLOCKS, 256, 0, s>>>(g, state, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mass_final_kernel<<<1, 32, 0, s>>>(g, partials, MASS_BLOCKS, out);
  return cudaGetLastError();
}

}  // namespace dgk
