// Consistent diffusion synthetic acceleration (paper App. B; used as stated in Sec. 4.1.1).
//
// The DSA correction solves the moment system obtained from the P1 ansatz
// delta f = delta rho + 3 v . delta J substituted into the upwind DG correction equation.
//
// 1D (App. B as printed), unknowns (drho, dJ) per cell:
//     D_C dJ - c1 D_J drho + Sigma_a drho = R,      c1 = sum_{v>0} w v
//     c2 D_C drho + (Sigma_t - 3 c3 D_J) dJ = 0,     c2 = sum w v^2, c3 = sum_{v>0} w v^3
// is block tridiagonal (4x4 blocks per cell) and is solved directly (block Thomas), as the paper
// solves 1D DSA with a direct solver.
//
// 2D: the same derivation in X-Y geometry gives, per cell, 12 unknowns (drho, dJx, dJy):
//     [Sigma_a - <|vx|>/2 DJx - <|vy|>/2 DJy] drho + 3<vx^2> DCx dJx + 3<vy^2> DCy dJy = R
//     <vx^2> DCx drho + [3<vx^2> Sigma_t - 3/2 <|vx|^3> DJx - 3/2 <vx^2|vy|> DJy] dJx = 0
//     <vy^2> DCy drho + [3<vy^2> Sigma_t - 3/2 <|vy|^3> DJy - 3/2 <vy^2|vx|> DJx] dJy = 0
// (<.> = quadrature sums).  On a uniform mesh D_C and D_J are geometry-only: per cell a 12x12
// diagonal block that depends on the cell's material, and four constant 12x12 neighbour blocks.
// The paper solves this with algebraic multigrid; here it is solved by flexible GMRES with an
// FP64 matrix-free operator, preconditioned by one geometric multigrid V-cycle in FP32:
// Galerkin coarse operators P^T A P built from the nested DG spaces (a coarse cell's Q^1
// functions restricted to its 2x2 children), red-black 12x12-block Gauss-Seidel smoothing, and
// the 1x1 coarsest level inverted exactly.  The preconditioner's precision affects only the
// iteration count; the FP64 residual decides convergence.
#include "common.cuh"

namespace rte {

constexpr int NB = 12;     // unknowns per cell (3 fields x 4 Q1 moments)
constexpr int NB2 = 144;

// ---- 1D local operators (orthonormal P1 basis, traces L=(1,-s3)/sqrt h, R=(1,s3)/sqrt h) -----
struct Ops1D {
  double DCd[4], DCw[4], DCe[4], DJd[4], DJw[4], DJe[4];  // 2x2 row-major
};

static Ops1D ops1d(double h) {
  const double s3 = std::sqrt(3.0), q = 1.0 / std::sqrt(h);
  const double L[2] = {q, -s3 * q}, R[2] = {q, s3 * q};
  Ops1D o{};
  for (int k = 0; k < 2; ++k)
    for (int l = 0; l < 2; ++l) {
      const double V = (k == 1 && l == 0) ? -2.0 * s3 / h : 0.0;  // -int phi_k' phi_l
      o.DCd[2 * k + l] = V + 0.5 * (R[k] * R[l] - L[k] * L[l]);
      o.DCw[2 * k + l] = -0.5 * L[k] * R[l];
      o.DCe[2 * k + l] = 0.5 * R[k] * L[l];
      o.DJd[2 * k + l] = -L[k] * L[l] - R[k] * R[l];
      o.DJw[2 * k + l] = L[k] * R[l];
      o.DJe[2 * k + l] = R[k] * L[l];
    }
  return o;
}

// The same operators on a non-uniform 1D mesh for a cell of width h with west / east neighbours
// of widths hw / he: the diagonal terms use h, each face coupling the traces of both cells.
static Ops1D ops1d_cell(double hw, double h, double he) {
  Ops1D o = ops1d(h);
  const double s3 = std::sqrt(3.0), q = 1.0 / std::sqrt(h), qw = 1.0 / std::sqrt(hw),
               qe = 1.0 / std::sqrt(he);
  const double L[2] = {q, -s3 * q}, R[2] = {q, s3 * q};
  const double Rw[2] = {qw, s3 * qw}, Le[2] = {qe, -s3 * qe};
  for (int k = 0; k < 2; ++k)
    for (int l = 0; l < 2; ++l) {
      o.DCw[2 * k + l] = -0.5 * L[k] * Rw[l];
      o.DCe[2 * k + l] = 0.5 * R[k] * Le[l];
      o.DJw[2 * k + l] = L[k] * Rw[l];
      o.DJe[2 * k + l] = R[k] * Le[l];
    }
  return o;
}

// 4x4 operator acting on the x-degree (k = a + 2b): (I_b (x) A)[a+2b][a'+2b'] = A[a][a'] d_bb'
static void kron_x(const double A[4], double out[16]) {
  for (int k = 0; k < 16; ++k) out[k] = 0.0;
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a)
      for (int a2 = 0; a2 < 2; ++a2) out[4 * (a + 2 * b) + (a2 + 2 * b)] = A[2 * a + a2];
}
static void kron_y(const double A[4], double out[16]) {
  for (int k = 0; k < 16; ++k) out[k] = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int b2 = 0; b2 < 2; ++b2) out[4 * (a + 2 * b) + (a + 2 * b2)] = A[2 * b + b2];
}

// 12x12 block from 4x4 x/y pieces; diag adds the sigma terms.
static void field_block(const DsaMoments& m, const double DCx[16], const double DJx[16],
                        const double DCy[16], const double DJy[16], double sa, double st,
                        bool diag, double out[NB2]) {
  for (int k = 0; k < NB2; ++k) out[k] = 0.0;
  auto put = [&](int fr, int fc, int r, int c, double v) { out[(4 * fr + r) * NB + 4 * fc + c] += v; };
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      const int e = 4 * r + c;
      const double I = (diag && r == c) ? 1.0 : 0.0;
      put(0, 0, r, c, -0.5 * m.abs_x * DJx[e] - 0.5 * m.abs_y * DJy[e] + sa * I);
      put(0, 1, r, c, 3.0 * m.xx * DCx[e]);
      put(0, 2, r, c, 3.0 * m.yy * DCy[e]);
      put(1, 0, r, c, m.xx * DCx[e]);
      put(1, 1, r, c, -1.5 * m.abs3_x * DJx[e] - 1.5 * m.xx_absy * DJy[e] + 3.0 * m.xx * st * I);
      put(2, 0, r, c, m.yy * DCy[e]);
      put(2, 2, r, c, -1.5 * m.abs3_y * DJy[e] - 1.5 * m.yy_absx * DJx[e] + 3.0 * m.yy * st * I);
    }
}

// ---- device helpers -------------------------------------------------------------------------

// ---- multigrid levels ----------------------------------------------------------------------------
//
// The Galerkin coarse operator P^T A P of this DG moment system is the same system on the coarse
// mesh: coarse Q^1 functions are continuous inside a coarse cell, so every term on an interior
// fine face (jumps, averages times jumps) vanishes, and the volume and coarse-face terms are those
// of the coarse mesh.  Only the cross-section terms change: Sigma becomes the projected mass
// matrix sum_children P_c^T (sigma_c I) P_c.  So each level has constant neighbour couplings (set
// by its cell size) and a 12x12 diagonal block per cell = geometric part + mass blocks.  Cross
// sections are cellwise constant, so a coarse cell whose children all share one material has that
// material's block (the projected mass of a constant is the constant times I); only cells on a
// material interface need their own.  Each level therefore stores a class per cell (material, or
// one of the level's mixed cells) and one diagonal block per (instance, class).
//
// The neighbour blocks act only through face traces: the west neighbour contributes
// L (x) (C_W t) with t = the neighbour's right-face traces of the three fields (2 values each),
// L = (1, -sqrt3)/sqrt(h_x) the own left-face values and C_W a 3x3 field coupling from the
// quadrature moments; east, south and north likewise.

constexpr int kMaxLevels = 16;
constexpr int kFuseCells = 1024;  // levels this small run inside one fused kernel per instance

// Row-major 3x3 field couplings of the W, E, S, N faces of one level, divided by the cell size
// normal to the face (h_x for W, E and h_y for S, N): the neighbour's face traces and the cell's own
// face values each carry a factor 1 / sqrt(h).  Entries (0,2), (1,2), (2,0), (2,1) of W and E and
// (0,1), (1,0), (1,2), (2,1) of S and N are zero (an x face couples J_y only to J_y, a y face J_x
// only to J_x); the trace products skip them.
struct Coup {
  float W[9], E[9], S[9], N[9];
};

struct LevelC {
  int nx, ny, nc, n_class;
  int n_pure;          // classes 0 .. n_pure - 1 are single-material cells (parity-block D)
  const int32_t* cls;  // [nc] class of each cell (material map at level 0)
  const float* diag;   // [B][n_class][144]
  const float* dinv;   // [B][n_class][144]
  Coup K;              // this level's face couplings
  float* x;            // per instance [2][3][half][4] (see lword)
  float* b;
  float* r;
};

struct Fine {  // level 0 in FP64, for the Krylov operator
  const double* off64;   // [4][144]
  const double* diag64;  // [B][n_mat][144]
  const int32_t* mat;
  int n_mat;
};

__device__ __forceinline__ bool nbr(int d, int i, int j, int nx, int ny, int& c2) {
  int ii = i, jj = j;
  if (d == 1) --ii;
  else if (d == 2) ++ii;
  else if (d == 3) --jj;
  else ++jj;
  if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) return false;
  c2 = jj * nx + ii;
  return true;
}

// y = A0 x in FP64 on the finest level.  One thread per (cell, row of its block).
__global__ void fine_apply64_kernel(Fine F, int nx, int ny, int B, const double* __restrict__ x,
                                    double* __restrict__ y, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int nc = nx * ny;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * NB) return;
  const int c = t / NB, row = t % NB;
  const int i = c % nx, j = c / nx;
  const double* xb = x + (size_t)b * nc * NB;
  const double* D = F.diag64 + ((size_t)b * F.n_mat + F.mat[c]) * NB2 + row * NB;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < NB; ++k) acc = fma(D[k], xb[(size_t)c * NB + k], acc);
  for (int d = 1; d <= 4; ++d) {
    int c2;
    if (!nbr(d, i, j, nx, ny, c2)) continue;
    const double* O = F.off64 + (d - 1) * NB2 + row * NB;
#pragma unroll
    for (int k = 0; k < NB; ++k) acc = fma(O[k], xb[(size_t)c2 * NB + k], acc);
  }
  y[(size_t)b * nc * NB + t] = acc;
}

__device__ __forceinline__ void load12(const float* p, float v[NB]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 u = q[k];
    v[4 * k] = u.x, v[4 * k + 1] = u.y, v[4 * k + 2] = u.z, v[4 * k + 3] = u.w;
  }
}

__device__ __forceinline__ void store12(float* p, const float v[NB]) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < 3; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// ---- level vectors in HBM ------------------------------------------------------------------------
// Per instance [2 colours][3 fields][half][4] floats, half = ceil(nc / 2): the cells of colour
// (i + j) & 1 in the order of c / 2 (which numbers each colour's cells without gaps for either parity
// of nx), each field's 4 moments one 16-byte word.  A warp updating consecutive cells of one colour
// then reads each field of their neighbours -- consecutive cells of the other colour -- as one
// contiguous span of 16-byte words, and writes its own cells the same way (a cell's 12 values side
// by side would put consecutive cells of a colour 96 bytes apart).
__host__ __device__ __forceinline__ int lhalf(int nc) { return (nc + 1) / 2; }
__host__ __device__ __forceinline__ size_t lstride(int nc) { return (size_t)24 * lhalf(nc); }
__device__ __forceinline__ size_t lword(int half, int c, int col, int f) {
  return ((size_t)(col * 3 + f) * half + (c >> 1)) * 4;
}
__device__ __forceinline__ int lcolour(int c, int nx) {
  const int j = c / nx;
  return (c - j * nx + j) & 1;
}
// the 12 values of cell c (colour col) of one instance's vector v
__device__ __forceinline__ void lload(const float* v, int half, int c, int col, float out[NB]) {
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float4 u = *reinterpret_cast<const float4*>(v + lword(half, c, col, f));
    out[4 * f] = u.x, out[4 * f + 1] = u.y, out[4 * f + 2] = u.z, out[4 * f + 3] = u.w;
  }
}
__device__ __forceinline__ void lstore(float* v, int half, int c, int col, const float in[NB]) {
#pragma unroll
  for (int f = 0; f < 3; ++f)
    *reinterpret_cast<float4*>(v + lword(half, c, col, f)) =
        make_float4(in[4 * f], in[4 * f + 1], in[4 * f + 2], in[4 * f + 3]);
}

// The coupling of one face neighbour to a cell, added to acc, from the neighbour's 12 values v via
// its traces on the shared face: west (its right-face traces, the cell's left-face values), east,
// south (traces expanded along x) and north.  t[f][q]: trace of field f, q the moment along the
// face; u = K t the field couplings; the cell's face values expand u into its moments (1, -+sqrt3).
__device__ __forceinline__ void side_x(const float* __restrict__ Km, float sg, const float v[NB],
                                       float acc[NB]) {
  const float s3 = 1.7320508075688772f;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float t0 = fmaf(sg * s3, v[1 + 2 * q], v[2 * q]);
    const float t1 = fmaf(sg * s3, v[5 + 2 * q], v[4 + 2 * q]);
    const float t2 = fmaf(sg * s3, v[9 + 2 * q], v[8 + 2 * q]);
    const float u[3] = {fmaf(Km[1], t1, Km[0] * t0), fmaf(Km[4], t1, Km[3] * t0), Km[8] * t2};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      acc[4 * f + 2 * q] += u[f];
      acc[4 * f + 1 + 2 * q] = fmaf(-sg * s3, u[f], acc[4 * f + 1 + 2 * q]);
    }
  }
}
__device__ __forceinline__ void side_y(const float* __restrict__ Km, float sg, const float v[NB],
                                       float acc[NB]) {
  const float s3 = 1.7320508075688772f;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float t0 = fmaf(sg * s3, v[q + 2], v[q]);
    const float t1 = fmaf(sg * s3, v[4 + q + 2], v[4 + q]);
    const float t2 = fmaf(sg * s3, v[8 + q + 2], v[8 + q]);
    const float u[3] = {fmaf(Km[2], t2, Km[0] * t0), Km[4] * t1, fmaf(Km[8], t2, Km[6] * t0)};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      acc[4 * f + q] += u[f];
      acc[4 * f + q + 2] = fmaf(-sg * s3, u[f], acc[4 * f + q + 2]);
    }
  }
}
// west: the neighbour's right-face trace a0 + sqrt3 a1, the cell's left-face values (1, -sqrt3)
__device__ __forceinline__ void side_w(const Coup& K, const float v[NB], float acc[NB]) {
  side_x(K.W, 1.f, v, acc);
}
__device__ __forceinline__ void side_e(const Coup& K, const float v[NB], float acc[NB]) {
  side_x(K.E, -1.f, v, acc);
}
__device__ __forceinline__ void side_s(const Coup& K, const float v[NB], float acc[NB]) {
  side_y(K.S, 1.f, v, acc);
}
__device__ __forceinline__ void side_n(const Coup& K, const float v[NB], float acc[NB]) {
  side_y(K.N, -1.f, v, acc);
}

// acc += sum over the existing face neighbours of their coupling to a cell; w, e, s, n point to the
// 12 values of the west, east, south and north neighbours (null where there is none), in shared
// memory or registers.
__device__ __forceinline__ void nbr_trace_sum_p(const Coup& K, const float* w, const float* e,
                                                const float* s, const float* n, float acc[NB]) {
  float v[NB];
  if (w) load12(w, v), side_w(K, v, acc);
  if (e) load12(e, v), side_e(K, v, acc);
  if (s) load12(s, v), side_s(K, v, acc);
  if (n) load12(n, v), side_n(K, v, acc);
}

// the same for cell (i, j) of one instance's level vector x in global memory (its neighbours have
// the other colour)
__device__ __forceinline__ void nbr_trace_sum(const Coup& K, const float* __restrict__ x, int half,
                                              int i, int j, int nx, int ny, float acc[NB]) {
  const int nc = 1 - ((i + j) & 1);
  float v[NB];
  if (i > 0) lload(x, half, j * nx + i - 1, nc, v), side_w(K, v, acc);
  if (i + 1 < nx) lload(x, half, j * nx + i + 1, nc, v), side_e(K, v, acc);
  if (j > 0) lload(x, half, (j - 1) * nx + i, nc, v), side_s(K, v, acc);
  if (j + 1 < ny) lload(x, half, (j + 1) * nx + i, nc, v), side_n(K, v, acc);
}

__device__ __forceinline__ void matvec12(const float* __restrict__ M, const float v[NB], float out[NB]) {
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NB; ++k) s = fmaf(M[r * NB + k], v[k], s);
    out[r] = s;
  }
}

// The 12 unknowns (field f, moment k = kx + 2 ky) of a cell have parities (kx xor [f = 1],
// ky xor [f = 2]) under the reflections x -> -x and y -> -y.  The diagonal block of a single-
// material cell (geometric part plus sigma I mass blocks) is invariant under both, so it couples only
// unknowns of equal parities: D and D^-1 are four 3 x 3 blocks, 36 of the 144 entries, the others
// exact zeros.  Each row is summed in matvec12's order over its nonzero entries.
__device__ __forceinline__ void matvec12_parity(const float* __restrict__ M, const float v[NB],
                                                float out[NB]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int px = p & 1, py = p >> 1;
    const int g[3] = {px + 2 * py, 5 - px + 2 * py, 10 + px - 2 * py};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 3; ++q) s = fmaf(M[g[a] * NB + g[q]], v[g[q]], s);
      out[g[a]] = s;
    }
  }
}

// D (or D^-1) of class k times v: the parity blocks for a single-material class, else dense
__device__ __forceinline__ void apply_block(const LevelC& L, const float* __restrict__ M, int k,
                                            const float v[NB], float out[NB]) {
  if (k < L.n_pure) matvec12_parity(M, v, out);
  else matvec12(M, v, out);
}

// one cell of a red-black block Gauss-Seidel half sweep: x_c = D_c^{-1} (b_c - sum_n O_n x_n);
// dinv_b: the instance's D^-1 blocks [n_class][144] (global memory, or a shared-memory copy)
__device__ __forceinline__ void rbgs_cell(const LevelC& L, int b, int c, const float* dinv_b) {
  const int i = c % L.nx, j = c / L.nx, col = (i + j) & 1, half = lhalf(L.nc);
  float* xb = L.x + (size_t)b * lstride(L.nc);
  float acc[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) acc[r] = 0.f;
  nbr_trace_sum(L.K, xb, half, i, j, L.nx, L.ny, acc);
  float res[NB];
  lload(L.b + (size_t)b * lstride(L.nc), half, c, col, res);
#pragma unroll
  for (int r = 0; r < NB; ++r) res[r] -= acc[r];
  float out[NB];
  const int k = L.cls[c];
  apply_block(L, dinv_b + (size_t)k * NB2, k, res, out);
  lstore(xb, half, c, col, out);
}

// one cell of r = b - A x
// the 12 residual values of cell c of instance b
__device__ __forceinline__ void residual_values(const LevelC& L, int b, int c, float bl[NB]) {
  const int i = c % L.nx, j = c / L.nx, col = (i + j) & 1, half = lhalf(L.nc);
  const size_t off = (size_t)b * lstride(L.nc);
  const float* xb = L.x + off;
  float xl[NB], acc[NB];
  lload(xb, half, c, col, xl);
  const int k = L.cls[c];
  apply_block(L, L.diag + ((size_t)b * L.n_class + k) * NB2, k, xl, acc);
  nbr_trace_sum(L.K, xb, half, i, j, L.nx, L.ny, acc);
  lload(L.b + off, half, c, col, bl);
#pragma unroll
  for (int q = 0; q < NB; ++q) bl[q] -= acc[q];
}

__device__ __forceinline__ void residual_cell(const LevelC& L, int b, int c) {
  float bl[NB];
  residual_values(L, b, c, bl);
  const int i = c % L.nx, j = c / L.nx;
  lstore(L.r + (size_t)b * lstride(L.nc), lhalf(L.nc), c, (i + j) & 1, bl);
}

// Prolongation coefficients: fine basis a_f in the coarse basis a_c restricted to child o (-1/+1):
// p[o][a_f][a_c] = int_child phi^C_{a_c} phi^f_{a_f}.
__host__ __device__ __forceinline__ float pcoef(int o, int af, int ac) {
  const float r2 = 0.70710678118654752f;  // 1/sqrt2
  if (af == 0 && ac == 0) return r2;
  if (af == 0 && ac == 1) return (o < 0 ? -1.f : 1.f) * 0.61237243569579452f;  // sqrt6/4
  if (af == 1 && ac == 1) return 0.5f * r2;
  return 0.f;
}

// P entry for child (dx, dy) mapping coarse local k_c to fine local k_f (same field).
__host__ __device__ __forceinline__ float pk(int dx, int dy, int kf, int kc) {
  return pcoef(dx ? 1 : -1, kf & 1, kc & 1) * pcoef(dy ? 1 : -1, kf >> 1, kc >> 1);
}

// one entry t = (C, row) of b_coarse = sum_children P_c^T r[c]
__device__ __forceinline__ void restrict_entry(const LevelC& F, const LevelC& Cl, int b, int t) {
  const int C = t / NB, row = t % NB, f = row / 4, kc = row % 4;
  const int I = C % Cl.nx, J = C / Cl.nx;
  const int fh = lhalf(F.nc);
  const float* rb = F.r + (size_t)b * lstride(F.nc);
  float s = 0.f;
  for (int dy = 0; dy < 2; ++dy)
    for (int dx = 0; dx < 2; ++dx) {
      const int c = (2 * J + dy) * F.nx + 2 * I + dx;
      const float* rv = rb + lword(fh, c, (dx + dy) & 1, f);   // (2I + dx) + (2J + dy) has dx + dy's parity
#pragma unroll
      for (int kf = 0; kf < 4; ++kf) s = fmaf(pk(dx, dy, kf, kc), rv[kf], s);
    }
  Cl.b[(size_t)b * lstride(Cl.nc) + lword(lhalf(Cl.nc), C, (I + J) & 1, f) + kc] = s;
}

// one entry t = (c, row) of x_fine += P_c x_coarse[C]
__device__ __forceinline__ void prolong_entry(const LevelC& F, const LevelC& Cl, int b, int t) {
  const int c = t / NB, row = t % NB, f = row / 4, kf = row % 4;
  const int i = c % F.nx, j = c / F.nx;
  const int C = (j / 2) * Cl.nx + i / 2, dx = i & 1, dy = j & 1;
  const float* xv = Cl.x + (size_t)b * lstride(Cl.nc) +
                    lword(lhalf(Cl.nc), C, (i / 2 + j / 2) & 1, f);
  float s = 0.f;
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) s = fmaf(pk(dx, dy, kf, kc), xv[kc], s);
  F.x[(size_t)b * lstride(F.nc) + lword(lhalf(F.nc), c, (i + j) & 1, f) + kf] += s;
}

constexpr int kSmemClasses = 8;  // a level with at most this many classes has its D^-1 blocks
                                 // staged in shared memory by the smoothing kernels

__global__ void rbgs_kernel(LevelC L, int color, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ float4 dsh4[kSmemClasses * NB2 / 4];
  const float* dg = L.dinv + (size_t)b * L.n_class * NB2;
  const bool dsm = L.n_class <= kSmemClasses;
  if (dsm) {
    for (int t = threadIdx.x; t < L.n_class * NB2 / 4; t += blockDim.x)
      dsh4[t] = reinterpret_cast<const float4*>(dg)[t];
    __syncthreads();
  }
  const int hx2 = (L.nx + 1) / 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= hx2 * L.ny) return;
  const int j = idx / hx2;
  const int i = 2 * (idx % hx2) + ((j + color) & 1);
  if (i >= L.nx) return;
  rbgs_cell(L, b, j * L.nx + i, dsm ? reinterpret_cast<const float*>(dsh4) : dg);
}

// The first half sweep of post-smoothing with the prolongation x += P x_coarse folded in.  That
// half sweep overwrites the cells of `color` without reading them, so their prolongation is never
// needed, and the other colour's cells enter only as its neighbours: each neighbour's 12 values are
// corrected in registers with prolong_entry's arithmetic (the same single rounding as the stored
// sum) and the stored x of the other colour is left as it was -- the next half sweep recomputes
// those cells from scratch.  Saves the separate pass of prolong_add_kernel over x; bit for bit the
// same results.
__device__ __forceinline__ void nbr_prolonged(const float* __restrict__ xb, int half, const LevelC& Cl,
                                              int b, int ii, int jj, int nx, float v[NB]) {
  lload(xb, half, jj * nx + ii, (ii + jj) & 1, v);
  const int C = (jj / 2) * Cl.nx + ii / 2, dx = ii & 1, dy = jj & 1;
  float xc[NB];
  lload(Cl.x + (size_t)b * lstride(Cl.nc), lhalf(Cl.nc), C, (ii / 2 + jj / 2) & 1, xc);
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int kf = 0; kf < 4; ++kf) {
      float s = 0.f;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) s = fmaf(pk(dx, dy, kf, kc), xc[4 * f + kc], s);
      v[4 * f + kf] += s;
    }
}

// cell (i, j) of `color` in that half sweep; dinv_b the instance's D^-1 blocks
__device__ __forceinline__ void rbgs_prolong_cell(const LevelC& L, const LevelC& Cl, int b, int i,
                                                  int j, int color, const float* dinv_b) {
  const int c = j * L.nx + i, half = lhalf(L.nc);
  float* xb = L.x + (size_t)b * lstride(L.nc);
  float vw[NB], ve[NB], vs[NB], vn[NB];
  if (i > 0) nbr_prolonged(xb, half, Cl, b, i - 1, j, L.nx, vw);
  if (i + 1 < L.nx) nbr_prolonged(xb, half, Cl, b, i + 1, j, L.nx, ve);
  if (j > 0) nbr_prolonged(xb, half, Cl, b, i, j - 1, L.nx, vs);
  if (j + 1 < L.ny) nbr_prolonged(xb, half, Cl, b, i, j + 1, L.nx, vn);
  float acc[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) acc[r] = 0.f;
  nbr_trace_sum_p(L.K, i > 0 ? vw : nullptr, i + 1 < L.nx ? ve : nullptr, j > 0 ? vs : nullptr,
                  j + 1 < L.ny ? vn : nullptr, acc);
  float res[NB];
  lload(L.b + (size_t)b * lstride(L.nc), half, c, color, res);
#pragma unroll
  for (int r = 0; r < NB; ++r) res[r] -= acc[r];
  float out[NB];
  const int k = L.cls[c];
  apply_block(L, dinv_b + (size_t)k * NB2, k, res, out);
  lstore(xb, half, c, color, out);
}

__global__ void rbgs_prolong_kernel(LevelC L, LevelC Cl, int color, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ float4 dsh4[kSmemClasses * NB2 / 4];
  const float* dg = L.dinv + (size_t)b * L.n_class * NB2;
  const bool dsm = L.n_class <= kSmemClasses;
  if (dsm) {
    for (int t = threadIdx.x; t < L.n_class * NB2 / 4; t += blockDim.x)
      dsh4[t] = reinterpret_cast<const float4*>(dg)[t];
    __syncthreads();
  }
  const int hx2 = (L.nx + 1) / 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= hx2 * L.ny) return;
  const int j = idx / hx2;
  const int i = 2 * (idx % hx2) + ((j + color) & 1);
  if (i >= L.nx) return;
  rbgs_prolong_cell(L, Cl, b, i, j, color, dsm ? reinterpret_cast<const float*>(dsh4) : dg);
}

// Red-black Gauss-Seidel with temporal blocking: H = 2 nu half sweeps of one level, colours c0,
// 1 - c0, c0, ..., on a 16 x 16 tile per CTA, in shared memory.  The CTA loads x and b on the tile
// and a halo of H cells, then half sweep h updates the cells of its colour within H - 1 - h cells
// of the tile (their neighbours are exact after half sweep h - 1 there), so after H half sweeps
// the tile holds exactly what H launches of rbgs_kernel give; only the tile is written, to xout
// (not to L.x, whose halo cells other CTAs are still reading).  One pass over x and b instead of
// H, for 1.4x the cell updates (the shrinking halo).  Each cell update is rbgs_cell's arithmetic
// in the same order, so results are bit for bit those of rbgs_kernel.
constexpr int kFT = 16;        // tile side
constexpr int kFusedMaxH = 8;  // half sweeps per launch at most (nu <= 4)

constexpr int kFusedClasses = kSmemClasses;

__host__ __device__ constexpr size_t fused_smem_bytes(int H) {
  return ((size_t)2 * (kFT + 2 * H) * (kFT + 2 * H) * NB + (size_t)kFusedClasses * NB2) * sizeof(float);
}

__global__ void __launch_bounds__(256) rbgs_fused_kernel(LevelC L, int H, int c0, float* xout,
                                                         const uint8_t* active) {
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  extern __shared__ float4 fsm4[];
  const int R = kFT + 2 * H;
  float* xs = reinterpret_cast<float*>(fsm4);  // [R * R][12] region, row-major
  float* bs = xs + (size_t)R * R * NB;
  float* ds = bs + (size_t)R * R * NB;         // [n_class][144] D^-1 blocks when few classes
  const bool dsm = L.n_class <= kFusedClasses;
  const float* dg = L.dinv + (size_t)b * L.n_class * NB2;
  if (dsm)
    for (int t = threadIdx.x; t < L.n_class * NB2 / 4; t += blockDim.x)
      reinterpret_cast<float4*>(ds)[t] = reinterpret_cast<const float4*>(dg)[t];
  const int i0 = blockIdx.x * kFT - H, j0 = blockIdx.y * kFT - H;  // region origin
  const int lh = lhalf(L.nc);
  const float* xg = L.x + (size_t)b * lstride(L.nc);
  const float* bg = L.b + (size_t)b * lstride(L.nc);
  float* xo = xout + (size_t)b * lstride(L.nc);
  for (int t = threadIdx.x; t < R * R * 3; t += blockDim.x) {
    const int cell = t / 3, q = t % 3, gi = i0 + cell % R, gj = j0 + cell / R;
    if (gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny) {
      const size_t g = lword(lh, gj * L.nx + gi, (gi + gj) & 1, q);
      reinterpret_cast<float4*>(xs + (size_t)cell * NB)[q] = *reinterpret_cast<const float4*>(xg + g);
      reinterpret_cast<float4*>(bs + (size_t)cell * NB)[q] = *reinterpret_cast<const float4*>(bg + g);
    }
  }
  __syncthreads();
  for (int h = 0; h < H; ++h) {
    const int color = (c0 + h) & 1, d = H - 1 - h;
    const int lo = H - d, W = kFT + 2 * d, half = (W + 1) / 2;  // region rows/cols [lo, lo + W)
    for (int t = threadIdx.x; t < W * half; t += blockDim.x) {
      const int rj = lo + t / half, gj = j0 + rj;
      // first column of this row with (gi + gj) % 2 == color, then every second one
      const int ri = lo + ((color - gj - (i0 + lo)) & 1) + 2 * (t % half), gi = i0 + ri;
      if (ri >= lo + W || gi < 0 || gi >= L.nx || gj < 0 || gj >= L.ny) continue;
      const int cell = rj * R + ri;
      float acc[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) acc[r] = 0.f;
      nbr_trace_sum_p(L.K, gi > 0 ? xs + (size_t)(cell - 1) * NB : nullptr,
                      gi + 1 < L.nx ? xs + (size_t)(cell + 1) * NB : nullptr,
                      gj > 0 ? xs + (size_t)(cell - R) * NB : nullptr,
                      gj + 1 < L.ny ? xs + (size_t)(cell + R) * NB : nullptr, acc);
      float res[NB];
      load12(bs + (size_t)cell * NB, res);
#pragma unroll
      for (int r = 0; r < NB; ++r) res[r] -= acc[r];
      float out[NB];
      const int k = L.cls[gj * L.nx + gi];
      apply_block(L, (dsm ? ds : dg) + (size_t)k * NB2, k, res, out);
      store12(xs + (size_t)cell * NB, out);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kFT * kFT * 3; t += blockDim.x) {
    const int cell = t / 3, q = t % 3, ri = H + cell % kFT, rj = H + cell / kFT;
    const int gi = i0 + ri, gj = j0 + rj;
    if (gi < L.nx && gj < L.ny)
      *reinterpret_cast<float4*>(xo + lword(lh, gj * L.nx + gi, (gi + gj) & 1, q)) =
          reinterpret_cast<const float4*>(xs + (size_t)(rj * R + ri) * NB)[q];
  }
}

// One red-black half sweep on 16 x 16 tiles: the CTA first loads the cells of the other colour
// on its tile and a one-cell halo into shared memory with coalesced 16-byte loads (each such cell
// once, instead of once per neighbour that reads it), then each of its 128 threads updates one
// cell of `color` from there.  Cells of `color` are only written and cells of the other colour
// only read, so the update is in place.  Same arithmetic as rbgs_kernel, bit for bit.
constexpr int kTT = 16;  // tile side

__global__ void __launch_bounds__(128) rbgs_tiled_kernel(LevelC L, int color, const uint8_t* active) {
  const int b = blockIdx.z;
  if (active && !active[b]) return;
  constexpr int R = kTT + 2;
  __shared__ float4 xs4[R * R * 3];
  __shared__ float4 dsh4[kSmemClasses * NB2 / 4];
  float* xs = reinterpret_cast<float*>(xs4);
  const int lh = lhalf(L.nc);
  float* xg = L.x + (size_t)b * lstride(L.nc);
  const int i0 = blockIdx.x * kTT - 1, j0 = blockIdx.y * kTT - 1;  // region origin
  for (int t = threadIdx.x; t < R * R * 3; t += blockDim.x) {
    const int cell = t / 3, q = t % 3, gi = i0 + cell % R, gj = j0 + cell / R;
    if (gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny && ((gi + gj) & 1) != color)
      xs4[t] = *reinterpret_cast<const float4*>(xg + lword(lh, gj * L.nx + gi, 1 - color, q));
  }
  const float* dg = L.dinv + (size_t)b * L.n_class * NB2;
  const bool dsm = L.n_class <= kSmemClasses;
  if (dsm)
    for (int t = threadIdx.x; t < L.n_class * NB2 / 4; t += blockDim.x)
      dsh4[t] = reinterpret_cast<const float4*>(dg)[t];
  __syncthreads();
  // thread k: tile row k / 8, the (k % 8)-th cell of `color` in that row
  const int rr = threadIdx.x >> 3, gj = j0 + 1 + rr;
  const int ci = 2 * (threadIdx.x & 7) + ((color - gj - (i0 + 1)) & 1), gi = i0 + 1 + ci;
  if (gi >= L.nx || gj >= L.ny) return;
  const int cell = (rr + 1) * R + ci + 1;
  float acc[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) acc[r] = 0.f;
  nbr_trace_sum_p(L.K, gi > 0 ? xs + (size_t)(cell - 1) * NB : nullptr,
                  gi + 1 < L.nx ? xs + (size_t)(cell + 1) * NB : nullptr,
                  gj > 0 ? xs + (size_t)(cell - R) * NB : nullptr,
                  gj + 1 < L.ny ? xs + (size_t)(cell + R) * NB : nullptr, acc);
  const int c = gj * L.nx + gi;
  float res[NB];
  lload(L.b + (size_t)b * lstride(L.nc), lh, c, color, res);
#pragma unroll
  for (int r = 0; r < NB; ++r) res[r] -= acc[r];
  float out[NB];
  const int k = L.cls[c];
  apply_block(L, (dsm ? reinterpret_cast<const float*>(dsh4) : dg) + (size_t)k * NB2, k, res, out);
  lstore(xg, lh, c, color, out);
}

__global__ void residual_kernel(LevelC L, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.nc) return;
  residual_cell(L, b, c);
}

// r = b - A x on level F and its restriction b_coarse = sum_children P_c^T r[c] in one pass: one
// thread per coarse cell computes its four children's residuals in registers (residual_cell's
// arithmetic) and sums each coarse entry over the children in restrict_entry's order, so the
// result is bit for bit that of residual_kernel followed by restrict_kernel without writing and
// re-reading the residual.
__device__ __forceinline__ void residual_restrict_cell(const LevelC& F, const LevelC& Cl, int b, int C) {
  const int I = C % Cl.nx, J = C / Cl.nx;
  float r[4][NB];
#pragma unroll
  for (int dy = 0; dy < 2; ++dy)
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) residual_values(F, b, (2 * J + dy) * F.nx + 2 * I + dx, r[2 * dy + dx]);
  float* bc = Cl.b + (size_t)b * lstride(Cl.nc);
  const int ch = lhalf(Cl.nc), ccol = (I + J) & 1;
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    float out[4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      float acc = 0.f;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
          for (int kf = 0; kf < 4; ++kf) acc = fmaf(pk(dx, dy, kf, kc), r[2 * dy + dx][4 * f + kf], acc);
      out[kc] = acc;
    }
    *reinterpret_cast<float4*>(bc + lword(ch, C, ccol, f)) = make_float4(out[0], out[1], out[2], out[3]);
  }
}

__global__ void residual_restrict_kernel(LevelC F, LevelC Cl, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= Cl.nc) return;
  residual_restrict_cell(F, Cl, b, C);
}

__global__ void restrict_kernel(LevelC F, LevelC Cl, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Cl.nc * NB) return;
  restrict_entry(F, Cl, b, t);
}

__global__ void prolong_add_kernel(LevelC F, LevelC Cl, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= F.nc * NB) return;
  prolong_entry(F, Cl, b, t);
}

struct CoarseArgs {
  int lc, nL, nu;
  LevelC lv[kMaxLevels];
};

// The V-cycle from level lc down to the coarsest and back, one CTA per instance; phases are
// separated by block barriers instead of launches.  lc is the first level with <= kFuseCells
// cells.  The barriers bound this kernel, so it takes the fine levels' shortcuts, each the same
// arithmetic as the phases it replaces: the first half sweep from x = 0 sets x_c = D_c^-1 b_c on
// the cells of colour 0 without clearing x (the cells of colour 1 are overwritten by the next half
// sweep before anything reads them); residual and restriction are one pass over the coarse cells
// (residual_restrict_cell); the prolongation is folded into the first half sweep of
// post-smoothing (rbgs_prolong_cell).
__global__ void __launch_bounds__(512) coarse_vcycle_kernel(const CoarseArgs A, const uint8_t* active) {
  const int b = blockIdx.x;
  if (active && !active[b]) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  auto half_sweep = [&](const LevelC& L, int color) {
    const int hx2 = (L.nx + 1) / 2;
    for (int idx = tid; idx < hx2 * L.ny; idx += nt) {
      const int j = idx / hx2, i = 2 * (idx % hx2) + ((j + color) & 1);
      if (i < L.nx) rbgs_cell(L, b, j * L.nx + i, L.dinv + (size_t)b * L.n_class * NB2);
    }
    __syncthreads();
  };
  // the first half sweep (colour 0) from x = 0: x_c = D_c^-1 b_c
  auto first_half = [&](const LevelC& L) {
    const float* dinv_b = L.dinv + (size_t)b * L.n_class * NB2;
    const size_t off = (size_t)b * lstride(L.nc);
    const int half = lhalf(L.nc), hx2 = (L.nx + 1) / 2;
    for (int idx = tid; idx < hx2 * L.ny; idx += nt) {
      const int j = idx / hx2, i = 2 * (idx % hx2) + (j & 1);
      if (i >= L.nx) continue;
      const int c = j * L.nx + i, k = L.cls[c];
      float v[NB], out[NB];
      lload(L.b + off, half, c, 0, v);
      apply_block(L, dinv_b + (size_t)k * NB2, k, v, out);
      lstore(L.x + off, half, c, 0, out);
    }
    __syncthreads();
  };
  int l = A.lc;
  for (;; ++l) {  // down
    const LevelC& L = A.lv[l];
    first_half(L);
    if (l == A.nL - 1) {  // coarsest: exact for one cell, else many sweeps
      if (L.nc > 1) {
        half_sweep(L, 1);
        for (int k = 1; k < 30; ++k) half_sweep(L, 0), half_sweep(L, 1);
      }
      break;
    }
    half_sweep(L, 1);
    for (int k = 1; k < A.nu; ++k) half_sweep(L, 0), half_sweep(L, 1);
    const LevelC& Cl = A.lv[l + 1];
    for (int C = tid; C < Cl.nc; C += nt) residual_restrict_cell(L, Cl, b, C);
    __syncthreads();
  }
  for (l = A.nL - 2; l >= A.lc; --l) {  // up
    const LevelC& L = A.lv[l];
    const float* dinv_b = L.dinv + (size_t)b * L.n_class * NB2;
    const int hx2 = (L.nx + 1) / 2;
    for (int idx = tid; idx < hx2 * L.ny; idx += nt) {   // colour 1, the prolongation folded in
      const int j = idx / hx2, i = 2 * (idx % hx2) + ((j + 1) & 1);
      if (i < L.nx) rbgs_prolong_cell(L, A.lv[l + 1], b, i, j, 1, dinv_b);
    }
    __syncthreads();
    half_sweep(L, 0);
    for (int k = 1; k < A.nu; ++k) half_sweep(L, 1), half_sweep(L, 0);
  }
}

// ---- set-up kernels: per (instance, class) mass blocks and diagonal blocks ---------------------

// Masses of level l per (instance, class): materials sigma I; mixed cells sum_children P^T M P with
// the children's masses taken from level l-1 by their classes.
// Mass blocks of every (instance, class) of level l, one thread per (instance, class, entry): a
// material class holds sigma_a I and sigma_t I; a mixed class of a coarse level the Galerkin
// projection sum over its 2 x 2 children of P_c^T M_child P_c (the children's blocks from level
// l - 1).  Each entry is summed over the children and the P coefficients in a fixed order.
__global__ void class_mass_kernel(int l, int n_mat, int n_class, int n_class_f, int nxf, int nxc,
                                  const int32_t* mixed, const int32_t* cls_f,
                                  const double* sigma_t, const double* sigma_s, int B,
                                  const double* Maf, const double* Mtf, double* Ma, double* Mt,
                                  const uint8_t* mask) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * n_class * 16) return;
  const int e = t % 16, bk = t / 16;
  const int b = bk / n_class, k = bk % n_class;
  if (mask && !mask[b]) return;
  const int r = e / 4, q = e % 4;
  double ma = 0.0, mt = 0.0;
  if (k < n_mat) {
    if (r == q) {
      const double st = sigma_t[b * n_mat + k];
      ma = st - sigma_s[b * n_mat + k];
      mt = st;
    }
  } else {
    const int C = mixed[k - n_mat];
    const int I = C % nxc, J = C / nxc;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int c = (2 * J + dy) * nxf + 2 * I + dx;
        const double* fa = Maf + ((size_t)b * n_class_f + cls_f[c]) * 16;
        const double* ft = Mtf + ((size_t)b * n_class_f + cls_f[c]) * 16;
        double sa = 0.0, stt = 0.0;
        for (int kk = 0; kk < 4; ++kk) {
          const double pr = pk(dx, dy, kk, r);
          if (pr == 0.0) continue;
          for (int ll = 0; ll < 4; ++ll) {
            const double pq = pk(dx, dy, ll, q);
            sa += pr * fa[4 * kk + ll] * pq;
            stt += pr * ft[4 * kk + ll] * pq;
          }
        }
        ma += sa;
        mt += stt;
      }
  }
  Ma[(size_t)bk * 16 + e] = ma;
  Mt[(size_t)bk * 16 + e] = mt;
}

// D = geo + blockdiag(Ma, 3<vx^2> Mt, 3<vy^2> Mt) per (instance, class); store D, D^{-1} (FP32)
// and, when diag64 != nullptr, D in FP64.  One warp per block: lane c < 24 holds column c of the
// augmented matrix [D | I] in registers, and the Gauss-Jordan elimination with partial pivoting of
// inv12 runs column-parallel (the pivot column's lane picks the pivot row and broadcasts the
// scaling and elimination factors); every element sees inv12's operations in inv12's order.
__global__ void class_diag_kernel(const double* geo, const double* Ma, const double* Mt, double cx,
                                  double cy, int n, float* diag, float* dinv, double* diag64,
                                  int n_class, const uint8_t* mask) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (t >= n) return;
  if (mask && !mask[t / n_class]) return;
  double col[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    double v = 0.0;
    if (lane < NB) {
      const int c = lane;
      v = geo[r * NB + c];
      const int fr = r / 4, fc = c / 4;
      if (fr == fc) {
        const double m = fr == 0 ? Ma[(size_t)t * 16 + 4 * (r % 4) + (c % 4)]
                                 : (fr == 1 ? cx : cy) * Mt[(size_t)t * 16 + 4 * (r % 4) + (c % 4)];
        v += m;
      }
      diag[(size_t)t * NB2 + r * NB + c] = (float)v;
      if (diag64) diag64[(size_t)t * NB2 + r * NB + c] = v;
    } else if (lane < 2 * NB) {
      v = r == lane - NB ? 1.0 : 0.0;
    }
    col[r] = v;
  }
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    // pivot row: the first largest |a[r][k]|, r >= k (lane k owns column k)
    int p = k;
    double best = fabs(col[k]);
#pragma unroll
    for (int r = k + 1; r < NB; ++r)
      if (fabs(col[r]) > best) best = fabs(col[r]), p = r;
    p = __shfl_sync(0xffffffffu, p, k);
    if (p != k) {
      double tk = col[k], tp = tk;
#pragma unroll
      for (int r = k + 1; r < NB; ++r) tp = r == p ? col[r] : tp;
#pragma unroll
      for (int r = k + 1; r < NB; ++r) col[r] = r == p ? tk : col[r];
      col[k] = tp;
    }
    const double piv = 1.0 / __shfl_sync(0xffffffffu, col[k], k);
    col[k] *= piv;
#pragma unroll
    for (int r = 0; r < NB; ++r)
      if (r != k) {
        const double f = __shfl_sync(0xffffffffu, col[r], k);
        col[r] -= f * col[k];
      }
  }
  if (lane >= NB && lane < 2 * NB)
#pragma unroll
    for (int r = 0; r < NB; ++r) dinv[(size_t)t * NB2 + r * NB + (lane - NB)] = (float)col[r];
}

// ---- vector helpers (FGMRES, FP64) ---------------------------------------------------------

__global__ void pack_rhs_kernel(const double* R, double* v, int nc, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * NB) return;
  const int c = t / NB, k = t % NB;
  v[(size_t)b * nc * NB + t] = k < 4 ? R[(size_t)b * nc * 4 + 4 * c + k] : 0.0;
}

__global__ void extract_rho_kernel(const double* x, double* drho, int nc, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc * 4) return;
  const int c = t / 4, k = t % 4;
  drho[(size_t)b * nc * 4 + t] = x[((size_t)b * nc + c) * NB + k];
}

// dots[b][i] = <V_i[b], w[b]> for i < k; one block per (i, b); fixed-order tree reduction.
__global__ void dots_kernel(const double* V, size_t vstride, const double* w, double* dots, int n,
                            int kmax, const uint8_t* active) {
  const int i = blockIdx.x, b = blockIdx.y;
  if (active && !active[b]) return;
  const double* vi = V + (size_t)i * vstride + (size_t)b * n;
  const double* wb = w + (size_t)b * n;
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) s = fma(vi[e], wb[e], s);
  __shared__ double sh[512];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) dots[(size_t)b * kmax + i] = sh[0];
}

// w[b] -= sum_{i<k} h[b][i] V_i[b]
__global__ void gs_update_kernel(const double* V, size_t vstride, double* w, const double* h,
                                 int n, int k, int kmax, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double s = w[(size_t)b * n + e];
    for (int i = 0; i < k; ++i) s -= h[(size_t)b * kmax + i] * V[(size_t)i * vstride + (size_t)b * n + e];
    w[(size_t)b * n + e] = s;
  }
}

// out[b] = alpha[b] * in[b]
__global__ void scale_kernel(const double* in, double* out, const double* alpha, int n, int kmax,
                             const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const double a = alpha[(size_t)b * kmax];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    out[(size_t)b * n + e] = a * in[(size_t)b * n + e];
}

// x[b] += sum_{i<k} y[b][i] Z_i[b]
__global__ void combine_kernel(const double* Z, size_t zstride, double* x, const double* y, int n,
                               int k, int kmax, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double s = x[(size_t)b * n + e];
    for (int i = 0; i < k; ++i) s += y[(size_t)b * kmax + i] * Z[(size_t)i * zstride + (size_t)b * n + e];
    x[(size_t)b * n + e] = s;
  }
}

// FP64 Krylov vectors ([nc][12] per instance) to and from FP32 level-0 vectors (colour-split)
__global__ void to32_kernel(const double* in, float* out, int nc, int nx, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int half = lhalf(nc);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc * NB; e += gridDim.x * blockDim.x) {
    const int c = e / NB, k = e % NB;
    out[(size_t)b * lstride(nc) + lword(half, c, lcolour(c, nx), k / 4) + k % 4] =
        (float)in[(size_t)b * nc * NB + e];
  }
}
__global__ void to64_kernel(const float* in, double* out, int nc, int nx, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int half = lhalf(nc);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc * NB; e += gridDim.x * blockDim.x) {
    const int c = e / NB, k = e % NB;
    out[(size_t)b * nc * NB + e] =
        (double)in[(size_t)b * lstride(nc) + lword(half, c, lcolour(c, nx), k / 4) + k % 4];
  }
}
__global__ void zero32_kernel(float* x, int per, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < per; e += gridDim.x * blockDim.x)
    x[(size_t)b * per + e] = 0.f;
}

// ---- 1D: block-tridiagonal direct solve ---------------------------------------------------------

// Per cell: unknowns u = (drho0, drho1, dJ0, dJ1).  Factor: Dp_c^{-1} and M_c = L_c Dp_{c-1}^{-1}.
__device__ void inv4d(const double* A, double* Ai) {
  double a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) a[r][c] = c < 4 ? A[4 * r + c] : (c - 4 == r ? 1.0 : 0.0);
  for (int k = 0; k < 4; ++k) {
    int p = k;
    for (int r = k + 1; r < 4; ++r)
      if (fabs(a[r][k]) > fabs(a[p][k])) p = r;
    if (p != k)
      for (int c = 0; c < 8; ++c) {
        double t = a[k][c];
        a[k][c] = a[p][c];
        a[p][c] = t;
      }
    const double piv = 1.0 / a[k][k];
    for (int c = 0; c < 8; ++c) a[k][c] *= piv;
    for (int r = 0; r < 4; ++r)
      if (r != k) {
        const double f = a[r][k];
        for (int c = 0; c < 8; ++c) a[r][c] -= f * a[k][c];
      }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) Ai[4 * r + c] = a[r][c + 4];
}

struct Blocks1D {
  const double *Dd, *Lw, *Ue;  // [nx][16] per cell: D without sigma terms; west / east couplings
};

// Block LU of the 1D consistent-DSA system, cell blocks over the unknowns (drho_0, drho_1,
// dJ_0, dJ_1): Sigma_a enters the (drho, drho) 2x2 and Sigma_t the (dJ, dJ) 2x2, each sigma I or,
// with cross sections linear across cells (matr non-null), the 2x2 of linear_sigma.
__global__ void dsa1d_factor_kernel(Blocks1D K, const double* sigma_t, const double* sigma_s,
                                    const int32_t* mat, const int32_t* matr, int nx, int n_mat,
                                    int B, double* Dpinv, double* Mfac, const uint8_t* mask) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (mask && !mask[b]) return;
  double Dp[16], Di[16], tmp[16];
  for (int c = 0; c < nx; ++c) {
    const int m = mat[c];
    double st = sigma_t[b * n_mat + m], sa = st - sigma_s[b * n_mat + m], to = 0.0, ao = 0.0;
    if (matr) {
      const int mr = matr[c];
      const double str = sigma_t[b * n_mat + mr], sar = str - sigma_s[b * n_mat + mr];
      linear_sigma(st, str, st, to);
      linear_sigma(sa, sar, sa, ao);
    }
    for (int e = 0; e < 16; ++e) Dp[e] = K.Dd[16 * c + e];
    Dp[0] += sa, Dp[5] += sa, Dp[10] += st, Dp[15] += st;
    Dp[1] += ao, Dp[4] += ao, Dp[11] += to, Dp[14] += to;
    double* Mc = Mfac + ((size_t)b * nx + c) * 16;
    if (c > 0) {
      const double* Dprev = Dpinv + ((size_t)b * nx + c - 1) * 16;
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) {
          double s = 0.0;
          for (int k = 0; k < 4; ++k) s += K.Lw[16 * c + 4 * r + k] * Dprev[4 * k + q];
          Mc[4 * r + q] = s;
        }
      for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) {
          double s = 0.0;
          for (int k = 0; k < 4; ++k) s += Mc[4 * r + k] * K.Ue[16 * (c - 1) + 4 * k + q];
          tmp[4 * r + q] = s;
        }
      for (int e = 0; e < 16; ++e) Dp[e] -= tmp[e];
    } else {
      for (int e = 0; e < 16; ++e) Mc[e] = 0.0;
    }
    inv4d(Dp, Di);
    for (int e = 0; e < 16; ++e) Dpinv[((size_t)b * nx + c) * 16 + e] = Di[e];
  }
}

__global__ void dsa1d_solve_kernel(Blocks1D K, const double* Dpinv, const double* Mfac,
                                   const double* R, double* drho, double* work, int nx, int B,
                                   const uint8_t* active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || (active && !active[b])) return;
  double* y = work + (size_t)b * nx * 4;
  double prev[4] = {0, 0, 0, 0};
  for (int c = 0; c < nx; ++c) {  // forward: y_c = b_c - M_c y_{c-1}
    const double bc[4] = {R[((size_t)b * nx + c) * 2], R[((size_t)b * nx + c) * 2 + 1], 0.0, 0.0};
    const double* Mc = Mfac + ((size_t)b * nx + c) * 16;
    for (int r = 0; r < 4; ++r) {
      double s = bc[r];
      for (int k = 0; k < 4; ++k) s -= Mc[4 * r + k] * prev[k];
      y[4 * c + r] = s;
    }
    for (int r = 0; r < 4; ++r) prev[r] = y[4 * c + r];
  }
  double next[4] = {0, 0, 0, 0};
  for (int c = nx - 1; c >= 0; --c) {  // backward: x_c = Dp_c^{-1} (y_c - U_c x_{c+1})
    double t[4];
    for (int r = 0; r < 4; ++r) {
      double s = y[4 * c + r];
      if (c < nx - 1)
        for (int k = 0; k < 4; ++k) s -= K.Ue[16 * c + 4 * r + k] * next[k];
      t[r] = s;
    }
    const double* Di = Dpinv + ((size_t)b * nx + c) * 16;
    for (int r = 0; r < 4; ++r) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += Di[4 * r + k] * t[k];
      next[r] = s;
    }
    drho[((size_t)b * nx + c) * 2] = next[0];
    drho[((size_t)b * nx + c) * 2 + 1] = next[1];
  }
}

// ---- state ------------------------------------------------------------------------------------

struct DsaState {
  int dim = 2;
  // 1D
  Blocks1D K1{};
  DevBuf<double> K1dev;                         // [3][nx][16] storage behind K1
  DevBuf<double> Dpinv, Mfac, work1;
  // 2D levels
  int n_levels = 0, lc = 0;                     // lc: first level of the fused coarse cycle
  std::vector<int> lnx, lny, ncls;
  std::vector<std::vector<int32_t>> cls_h, mixed_h;
  DevBuf<double> off64, diag64;                 // level 0 in FP64 (Krylov operator)
  std::vector<DevBuf<int32_t>*> cls, mixed;     // class per cell; mixed cells of each level
  std::vector<DevBuf<double>*> geo64;           // [144] per level
  std::vector<DevBuf<double>*> Ma, Mt;          // [B][n_class][16] per level
  std::vector<DevBuf<float>*> diag32, dinv32;   // [B][n_class][144] per level
  std::vector<DevBuf<float>*> xl, bl, rl;       // per level FP32 vectors
  DevBuf<float> xtot, borig;                    // stationary multigrid accumulator and rhs
  int m = 20;                                   // FGMRES restart length
  DevBuf<double> V, Z, w, xs;                   // Krylov bases and work
  DevBuf<double> dots_dev;
  template <class T>
  static void del(std::vector<T*>& v) {
    for (auto* p : v) delete p;
    v.clear();
  }
  ~DsaState() {
    del(cls), del(mixed), del(geo64), del(Ma), del(Mt), del(diag32), del(dinv32), del(xl), del(bl), del(rl);
  }
};

void dsa_state_free(DsaState* s) { delete s; }

static Fine fine_of(rte_batch_t bt) {
  DsaState* s = bt->dsa;
  return Fine{s->off64.p, s->diag64.p, bt->disc->mat_id.p, bt->disc->n_mat};
}

static Coup couplings(const DsaMoments& m, double hx, double hy);

static LevelC lvl_of(rte_batch_t bt, int l) {
  DsaState* s = bt->dsa;
  const rte_disc_s* d = bt->disc;
  LevelC L{};
  L.nx = s->lnx[l], L.ny = s->lny[l], L.nc = L.nx * L.ny, L.n_class = s->ncls[l];
  L.n_pure = d->n_mat;
  L.cls = s->cls[l]->p;
  L.diag = s->diag32[l]->p, L.dinv = s->dinv32[l]->p;
  L.K = couplings(d->mom, d->hx * (1 << l), d->hy * (1 << l));
  L.x = s->xl[l]->p, L.b = s->bl[l]->p, L.r = s->rl[l]->p;
  return L;
}

// constant neighbour blocks (FP64, for the Krylov operator) and geometric diagonal of a level
static void level_blocks(const DsaMoments& mom, double hx, double hy, double off[4 * NB2],
                         double geo[NB2]) {
  const Ops1D ox = ops1d(hx), oy = ops1d(hy);
  double DCx[3][16], DJx[3][16], DCy[3][16], DJy[3][16], Zr[16] = {0};
  kron_x(ox.DCd, DCx[0]), kron_x(ox.DCw, DCx[1]), kron_x(ox.DCe, DCx[2]);
  kron_x(ox.DJd, DJx[0]), kron_x(ox.DJw, DJx[1]), kron_x(ox.DJe, DJx[2]);
  kron_y(oy.DCd, DCy[0]), kron_y(oy.DCw, DCy[1]), kron_y(oy.DCe, DCy[2]);
  kron_y(oy.DJd, DJy[0]), kron_y(oy.DJw, DJy[1]), kron_y(oy.DJe, DJy[2]);
  field_block(mom, DCx[1], DJx[1], Zr, Zr, 0, 0, false, &off[0 * NB2]);  // W
  field_block(mom, DCx[2], DJx[2], Zr, Zr, 0, 0, false, &off[1 * NB2]);  // E
  field_block(mom, Zr, Zr, DCy[1], DJy[1], 0, 0, false, &off[2 * NB2]);  // S
  field_block(mom, Zr, Zr, DCy[2], DJy[2], 0, 0, false, &off[3 * NB2]);  // N
  field_block(mom, DCx[0], DJx[0], DCy[0], DJy[0], 0.0, 0.0, true, geo);
}

// field couplings of the trace form of the neighbour blocks on cells of size hx x hy: the
// quadrature moments' 3 x 3 couplings divided by the cell size normal to the face
static Coup couplings(const DsaMoments& m, double hx, double hy) {
  Coup K{};
  const double W[9] = {-0.5 * m.abs_x, -1.5 * m.xx, 0.0,
                       -0.5 * m.xx, -1.5 * m.abs3_x, 0.0,
                       0.0, 0.0, -1.5 * m.yy_absx};
  const double E[9] = {-0.5 * m.abs_x, 1.5 * m.xx, 0.0,
                       0.5 * m.xx, -1.5 * m.abs3_x, 0.0,
                       0.0, 0.0, -1.5 * m.yy_absx};
  const double S[9] = {-0.5 * m.abs_y, 0.0, -1.5 * m.yy,
                       0.0, -1.5 * m.xx_absy, 0.0,
                       -0.5 * m.yy, 0.0, -1.5 * m.abs3_y};
  const double N[9] = {-0.5 * m.abs_y, 0.0, 1.5 * m.yy,
                       0.0, -1.5 * m.xx_absy, 0.0,
                       0.5 * m.yy, 0.0, -1.5 * m.abs3_y};
  for (int k = 0; k < 9; ++k) {
    K.W[k] = (float)(W[k] / hx), K.E[k] = (float)(E[k] / hx);
    K.S[k] = (float)(S[k] / hy), K.N[k] = (float)(N[k] / hy);
  }
  return K;
}

template <class T>
static int upload(DevBuf<T>& buf, const std::vector<T>& h) {
  RTE_TRY(buf.alloc(h.size()));
  if (!h.empty())
    RTE_CUDA_TRY(cudaMemcpy(buf.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return RTE_OK;
}

// Levels, class tables and buffers: built once per batch (the material map is fixed).
static int dsa_build_levels(rte_batch_t bt) {
  const rte_disc_s* d = bt->disc;
  const int B = bt->B;
  DsaState* s = bt->dsa;
  s->lnx.push_back(d->nx);
  s->lny.push_back(d->ny);
  while (s->lnx.back() % 2 == 0 && s->lny.back() % 2 == 0 && s->lnx.back() * s->lny.back() > 1 &&
         (int)s->lnx.size() < kMaxLevels) {
    s->lnx.push_back(s->lnx.back() / 2);
    s->lny.push_back(s->lny.back() / 2);
  }
  s->n_levels = (int)s->lnx.size();
  s->lc = s->n_levels - 1;
  while (s->lc > 0 && s->lnx[s->lc - 1] * s->lny[s->lc - 1] <= kFuseCells) --s->lc;
  // (Running the whole cycle fused, one 512-thread CTA per instance, was measured slower than
  // level-by-level launches for the fine levels even with an instance per SM: 152 lattice
  // instances, DSA share 16% vs 14.5% of a step.)
  for (int l = 0; l < s->n_levels; ++l) {
    const int nx = s->lnx[l], ny = s->lny[l], nc = nx * ny;
    std::vector<int32_t> cls(nc), mixed;
    if (l == 0) {
      cls = d->mat_host;
    } else {
      const auto& cf = s->cls_h[l - 1];
      const int nxf = s->lnx[l - 1];
      for (int C = 0; C < nc; ++C) {
        const int I = C % nx, J = C / nx;
        int k0 = -1;
        bool pure = true;
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) {
            const int k = cf[(2 * J + dy) * nxf + 2 * I + dx];
            if (k >= d->n_mat) pure = false;
            if (k0 < 0) k0 = k;
            else if (k != k0) pure = false;
          }
        if (pure) cls[C] = k0;
        else cls[C] = d->n_mat + (int)mixed.size(), mixed.push_back(C);
      }
    }
    s->ncls.push_back(d->n_mat + (int)mixed.size());
    s->cls_h.push_back(cls);
    s->mixed_h.push_back(mixed);
    s->cls.push_back(new DevBuf<int32_t>());
    RTE_TRY(upload(*s->cls.back(), cls));
    s->mixed.push_back(new DevBuf<int32_t>());
    RTE_TRY(upload(*s->mixed.back(), mixed));
    std::vector<double> off(4 * NB2), geo(NB2);
    level_blocks(d->mom, d->hx * (1 << l), d->hy * (1 << l), off.data(), geo.data());
    if (l == 0) RTE_TRY(upload(s->off64, off));
    s->geo64.push_back(new DevBuf<double>());
    RTE_TRY(upload(*s->geo64.back(), geo));
    const size_t ncl = (size_t)B * s->ncls[l];
    for (auto* v : {&s->Ma, &s->Mt}) {
      v->push_back(new DevBuf<double>());
      RTE_TRY(v->back()->alloc(ncl * 16));
    }
    for (auto* v : {&s->diag32, &s->dinv32}) {
      v->push_back(new DevBuf<float>());
      RTE_TRY(v->back()->alloc(ncl * NB2));
    }
    for (auto* v : {&s->xl, &s->bl, &s->rl}) {
      v->push_back(new DevBuf<float>());
      RTE_TRY(v->back()->alloc((size_t)B * lstride(nc)));
    }
  }
  RTE_TRY(s->diag64.alloc((size_t)B * d->n_mat * NB2));
  const size_t n = (size_t)B * lstride(d->n_cells);
  RTE_TRY(s->xtot.alloc(n));
  RTE_TRY(s->borig.alloc(n));
  return RTE_OK;
}

// FGMRES bases and work vectors, allocated on the first Krylov solve of the batch
static int dsa_krylov_alloc(rte_batch_t bt) {
  DsaState* s = bt->dsa;
  if (s->V.p) return RTE_OK;
  const size_t n = (size_t)bt->B * bt->disc->n_cells * NB;
  RTE_TRY(s->V.alloc((size_t)(s->m + 1) * n));
  RTE_TRY(s->Z.alloc((size_t)s->m * n));
  RTE_TRY(s->w.alloc(n));
  RTE_TRY(s->xs.alloc(n));
  RTE_TRY(s->dots_dev.alloc((size_t)bt->B * (s->m + 1)));
  return RTE_OK;
}

// device bytes held by the batch's DSA state
size_t dsa_bytes(const rte_batch_s* b) {
  const DsaState* s = b->dsa;
  if (!s) return 0;
  size_t t = 0;
  auto add = [&](size_t n, size_t e) { t += n * e; };
  add(s->Dpinv.n + s->Mfac.n + s->work1.n + s->K1dev.n, 8);
  add(s->off64.n + s->diag64.n + s->V.n + s->Z.n + s->w.n + s->xs.n + s->dots_dev.n, 8);
  add(s->xtot.n + s->borig.n, 4);
  for (size_t l = 0; l < s->Ma.size(); ++l) {
    add(s->Ma[l]->n + s->Mt[l]->n + s->geo64[l]->n, 8);
    add(s->diag32[l]->n + s->dinv32[l]->n + s->xl[l]->n + s->bl[l]->n + s->rl[l]->n, 4);
    add(s->cls[l]->n + s->mixed[l]->n, 4);
  }
  return t;
}

int dsa_setup(rte_batch_t bt, cudaStream_t st, const uint8_t* mask) {
  const rte_disc_s* d = bt->disc;
  const int B = bt->B;
  if (!bt->dsa) bt->dsa = new DsaState();
  DsaState* s = bt->dsa;
  s->dim = d->dim;
  if (d->dim == 1) {
    // App. B constants from the S_N rule
    double c1 = 0, c2 = 0, c3 = 0;
    for (int j = 0; j < d->n_angles; ++j) {
      const double v = d->v[3 * j], w = d->w[j];
      c2 += w * v * v;
      if (v > 0) c1 += w * v, c3 += w * v * v * v;
    }
    auto fill = [&](double* out, const double* DC, const double* DJ) {
      // rows (rho0, rho1, J0, J1): [[-c1 DJ, DC], [c2 DC, -3 c3 DJ]]
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
          out[4 * r + c] = -c1 * DJ[2 * r + c];
          out[4 * r + c + 2] = DC[2 * r + c];
          out[4 * (r + 2) + c] = c2 * DC[2 * r + c];
          out[4 * (r + 2) + c + 2] = -3.0 * c3 * DJ[2 * r + c];
        }
    };
    if (!s->K1dev.p) {  // per-cell blocks from the cell widths (fixed per discretisation)
      const int nx = d->nx;
      std::vector<double> K((size_t)3 * nx * 16);
      for (int c = 0; c < nx; ++c) {
        const double h = d->dx[c];
        const Ops1D o = ops1d_cell(c > 0 ? d->dx[c - 1] : h, h, c + 1 < nx ? d->dx[c + 1] : h);
        fill(&K[(size_t)16 * c], o.DCd, o.DJd);
        fill(&K[(size_t)16 * (nx + c)], o.DCw, o.DJw);
        fill(&K[(size_t)16 * (2 * nx + c)], o.DCe, o.DJe);
      }
      RTE_TRY(upload(s->K1dev, K));
      s->K1 = Blocks1D{s->K1dev.p, s->K1dev.p + (size_t)16 * nx, s->K1dev.p + (size_t)32 * nx};
    }
    if (!s->Dpinv.p) {
      RTE_TRY(s->Dpinv.alloc((size_t)B * d->nx * 16));
      RTE_TRY(s->Mfac.alloc((size_t)B * d->nx * 16));
      RTE_TRY(s->work1.alloc((size_t)B * d->nx * 4));
    }
    dsa1d_factor_kernel<<<(B + 63) / 64, 64, 0, st>>>(s->K1, bt->sigma_t.p, bt->sigma_s.p,
                                                      d->mat_id.p, d->mat_r.p, d->nx, d->n_mat, B,
                                                      s->Dpinv.p, s->Mfac.p, mask); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
  }
  if (s->n_levels == 0) RTE_TRY(dsa_build_levels(bt));
  // per parameter set: masses and diagonal blocks of every (instance, class), level by level
  for (int l = 0; l < s->n_levels; ++l) {
    const int n = B * s->ncls[l];
    class_mass_kernel<<<(16 * n + 127) / 128, 128, 0, st>>>(
        l, d->n_mat, s->ncls[l], l ? s->ncls[l - 1] : 0, l ? s->lnx[l - 1] : 0, s->lnx[l],
        s->mixed[l]->p, l ? s->cls[l - 1]->p : nullptr, bt->sigma_t.p, bt->sigma_s.p, B,
        l ? s->Ma[l - 1]->p : nullptr, l ? s->Mt[l - 1]->p : nullptr, s->Ma[l]->p, s->Mt[l]->p,
        mask); RTE_NOTE_LAUNCH();
    class_diag_kernel<<<(n + 3) / 4, 128, 0, st>>>(s->geo64[l]->p, s->Ma[l]->p, s->Mt[l]->p,
                                                    3.0 * d->mom.xx, 3.0 * d->mom.yy, n,
                                                    s->diag32[l]->p, s->dinv32[l]->p,
                                                    l == 0 ? s->diag64.p : nullptr, s->ncls[l],
                                                    mask); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
  }
  return RTE_OK;
}

// One V-cycle from level l: x_l approximately solves A_l x = b_l (x_l starts at zero).
// Opt-in to the temporally blocked smoother's shared memory once per device.
static int fused_smem_attr(size_t bytes) {
  static size_t done[64] = {};
  int dev = 0;
  RTE_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(RTE_EINVAL, "device index too large");
  if (done[dev] >= bytes) return RTE_OK;
  const size_t want = fused_smem_bytes(kFusedMaxH);
  RTE_CUDA_TRY(cudaFuncSetAttribute(rbgs_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)want));
  done[dev] = want;
  return RTE_OK;
}

// first_done: level l's x holds the first half sweep of pre-smoothing from x = 0 already (colour 0
// cells set, colour 1 cells stale; pack_first_half_kernel), so the cycle neither clears x nor repeats
// that half sweep.  Only with the one-launch-per-half-sweep smoother forms.
static int vcycle(rte_batch_t bt, int l, const uint8_t* active, cudaStream_t st, int nu,
                  bool first_done = false) {
  DsaState* s = bt->dsa;
  const int B = bt->B;
  if (l >= s->lc) {  // the rest of the cycle in one launch, one CTA per instance
    CoarseArgs A{};
    A.lc = l, A.nL = s->n_levels, A.nu = nu;
    for (int k = 0; k < s->n_levels; ++k) A.lv[k] = lvl_of(bt, k);
    coarse_vcycle_kernel<<<B, 512, 0, st>>>(A, active); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
  }
  // the blocked smoother writes the level's residual buffer and then swaps it with x, so every
  // LevelC is re-read after a step that may have swapped them
  LevelC L = lvl_of(bt, l);
  if (!first_done) RTE_CUDA_TRY(cudaMemsetAsync(L.x, 0, sizeof(float) * (size_t)B * lstride(L.nc), st));
  const int ncol = ((L.nx + 1) / 2) * L.ny;
  const dim3 gcol((ncol + 127) / 128, B);
  const dim3 gtile((L.nx + kTT - 1) / kTT, (L.ny + kTT - 1) / kTT, B);
  auto smooth = [&](int c0) {
    if (bt->dsa_tiled) {
      rbgs_tiled_kernel<<<gtile, 128, 0, st>>>(L, c0, active); RTE_NOTE_LAUNCH();
      rbgs_tiled_kernel<<<gtile, 128, 0, st>>>(L, 1 - c0, active); RTE_NOTE_LAUNCH();
    } else {
      rbgs_kernel<<<gcol, 128, 0, st>>>(L, c0, active); RTE_NOTE_LAUNCH();
      rbgs_kernel<<<gcol, 128, 0, st>>>(L, 1 - c0, active); RTE_NOTE_LAUNCH();
    }
  };
  // nu sweeps starting with colour c0: one temporally blocked launch, or 2 nu launches
  const bool blocked = bt->dsa_blocking && 2 * nu <= kFusedMaxH;
  // pro: the coarse level whose prolongation is folded into the first half sweep (global form)
  auto smooth_nu = [&](int c0, const LevelC* pro) -> int {
    if (blocked) {
      const size_t bytes = fused_smem_bytes(2 * nu);
      RTE_TRY(fused_smem_attr(bytes));
      rbgs_fused_kernel<<<dim3((L.nx + kFT - 1) / kFT, (L.ny + kFT - 1) / kFT, B), 256, bytes, st>>>(
          L, 2 * nu, c0, L.r, active); RTE_NOTE_LAUNCH();
      std::swap(s->xl[l], s->rl[l]);  // the smoothed iterate is now the level's x
      L = lvl_of(bt, l);
    } else if (pro) {
      rbgs_prolong_kernel<<<gcol, 128, 0, st>>>(L, *pro, c0, active); RTE_NOTE_LAUNCH();
      rbgs_kernel<<<gcol, 128, 0, st>>>(L, 1 - c0, active); RTE_NOTE_LAUNCH();
      for (int k = 1; k < nu; ++k) smooth(c0);
    } else {
      for (int k = 0; k < nu; ++k) smooth(c0);
    }
    return RTE_OK;
  };
  if (first_done) {   // the rest of the first sweep (colour 1), then nu - 1 full sweeps
    if (bt->dsa_tiled) {
      rbgs_tiled_kernel<<<gtile, 128, 0, st>>>(L, 1, active); RTE_NOTE_LAUNCH();
    } else {
      rbgs_kernel<<<gcol, 128, 0, st>>>(L, 1, active); RTE_NOTE_LAUNCH();
    }
    for (int k = 1; k < nu; ++k) smooth(0);
  } else {
    RTE_TRY(smooth_nu(0, nullptr));
  }
  LevelC Cl = lvl_of(bt, l + 1);
  residual_restrict_kernel<<<dim3((Cl.nc + 127) / 128, B), 128, 0, st>>>(L, Cl, active); RTE_NOTE_LAUNCH();
  RTE_TRY(vcycle(bt, l + 1, active, st, nu));
  Cl = lvl_of(bt, l + 1);
  const bool fold = !blocked && !bt->dsa_tiled;  // the global form folds the prolongation in
  if (!fold) {
    prolong_add_kernel<<<dim3((L.nc * NB + 255) / 256, B), 256, 0, st>>>(L, Cl, active); RTE_NOTE_LAUNCH();
  }
  RTE_TRY(smooth_nu(1, fold ? &Cl : nullptr));
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

// R (FP64, 4 moments per cell) into a level-0 vector: the delta-rho field, the current fields zero.
__global__ void pack_rhs32_kernel(const double* R, float* v, int nc, int nx, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double* rc = R + ((size_t)b * nc + c) * 4;
  float u[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) u[k] = k < 4 ? (float)rc[k] : 0.f;
  lstore(v + (size_t)b * lstride(nc), lhalf(nc), c, lcolour(c, nx), u);
}

// The right-hand side R (FP64, 4 moments per cell) packed into level 0's b (the delta-rho block; the
// current blocks are zero) together with the first half sweep of pre-smoothing from x = 0: every
// neighbour of a cell of colour 0 is then zero, so that half sweep sets x_c = D_c^-1 b_c -- the
// same operations, in the same order, as rbgs_cell with zero neighbours, bit for bit.  The cells of
// colour 1 are left as they are: the next half sweep overwrites them without reading them.  Saves
// the separate pass that cleared x and one half sweep's neighbour reads.
__global__ void pack_first_half_kernel(LevelC L, const double* __restrict__ R, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  __shared__ float4 dsh4[kSmemClasses * NB2 / 4];
  const float* dg = L.dinv + (size_t)b * L.n_class * NB2;
  const bool dsm = L.n_class <= kSmemClasses;
  if (dsm) {
    for (int t = threadIdx.x; t < L.n_class * NB2 / 4; t += blockDim.x)
      dsh4[t] = reinterpret_cast<const float4*>(dg)[t];
    __syncthreads();
  }
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.nc) return;
  const double* rc = R + ((size_t)b * L.nc + c) * 4;
  float v[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) v[k] = k < 4 ? (float)rc[k] : 0.f;
  const int i = c % L.nx, j = c / L.nx, col = (i + j) & 1, half = lhalf(L.nc);
  lstore(L.b + (size_t)b * lstride(L.nc), half, c, col, v);
  if (col != 0) return;
  float out[NB];
  const int k = L.cls[c];
  apply_block(L, (dsm ? reinterpret_cast<const float*>(dsh4) : dg) + (size_t)k * NB2, k, v, out);
  lstore(L.x + (size_t)b * lstride(L.nc), half, c, col, out);
}

__global__ void add32_kernel(const float* x, float* y, int per, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < per; e += gridDim.x * blockDim.x)
    y[(size_t)b * per + e] += x[(size_t)b * per + e];
}

// the delta-rho field of a level-0 vector, in FP64 (4 moments per cell)
__global__ void extract_rho32_kernel(const float* x, double* drho, int nc, int nx,
                                     const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const float4 u = *reinterpret_cast<const float4*>(x + (size_t)b * lstride(nc) +
                                                    lword(lhalf(nc), c, lcolour(c, nx), 0));
  double2* o = reinterpret_cast<double2*>(drho + ((size_t)b * nc + c) * 4);
  o[0] = make_double2((double)u.x, (double)u.y);
  o[1] = make_double2((double)u.z, (double)u.w);
}

// out = base + the delta-rho field of a level-0 vector (FP64), for the instances in `active`: the
// SI update after a DSA correction in the pass that reads the correction (extract_rho32_kernel
// followed by the addition, bit for bit)
__global__ void extract_add32_kernel(const float* x, const double* __restrict__ base, double* out,
                                     int nc, int nx, const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const float4 u = *reinterpret_cast<const float4*>(x + (size_t)b * lstride(nc) +
                                                    lword(lhalf(nc), c, lcolour(c, nx), 0));
  const size_t o = ((size_t)b * nc + c) * 4;
  const double2 b01 = reinterpret_cast<const double2*>(base + o)[0];
  const double2 b23 = reinterpret_cast<const double2*>(base + o)[1];
  double2* w = reinterpret_cast<double2*>(out + o);
  w[0] = make_double2(b01.x + (double)u.x, b01.y + (double)u.y);
  w[1] = make_double2(b23.x + (double)u.z, b23.y + (double)u.w);
}

// residual on level 0 against an explicit right-hand side and iterate: r0 = borig - A0 xtot
__global__ void residual_ext_kernel(LevelC L, const float* bvec, const float* xv, float* r,
                                    const uint8_t* active) {
  const int b = blockIdx.y;
  if (active && !active[b]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.nc) return;
  LevelC M = L;
  M.b = const_cast<float*>(bvec), M.x = const_cast<float*>(xv), M.r = r;
  residual_cell(M, b, c);
}

// Stationary multigrid: k V-cycles on the FP32 system, x <- x + V(b - A x), no host round trip.
// With base != nullptr (one cycle only) the result is not stored as drho but added to base:
// drho[b] = base[b] + delta rho, extract_add32_kernel (the SI update rho^(l) = rho^(l,*) + delta rho
// of Alg. 1 in the same pass).
static int dsa2d_vcycles(rte_batch_t bt, const double* R, double* drho, int k,
                         const uint8_t* active, cudaStream_t st, const double* base = nullptr) {
  DsaState* s = bt->dsa;
  const int B = bt->B, nc = bt->disc->n_cells, nx = bt->disc->nx;
  const size_t per = lstride(nc);
  const dim3 gv((nc + 255) / 256, B), gvc((unsigned)std::min<size_t>((per + 255) / 256, 1024), B);
  if (k == 1) {
    // one cycle: pack the right-hand side straight into level 0 and read the result from there; with
    // a one-launch-per-half-sweep smoother the packing also does the first half sweep
    const bool fuse = !bt->dsa_blocking && s->lc > 0;
    if (fuse) {
      pack_first_half_kernel<<<dim3((nc + 127) / 128, B), 128, 0, st>>>(lvl_of(bt, 0), R, active); RTE_NOTE_LAUNCH();
    } else {
      pack_rhs32_kernel<<<gv, 256, 0, st>>>(R, s->bl[0]->p, nc, nx, active); RTE_NOTE_LAUNCH();
    }
    RTE_TRY(vcycle(bt, 0, active, st, bt->dsa_nu, fuse));
    if (base) {
      extract_add32_kernel<<<gv, 256, 0, st>>>(s->xl[0]->p, base, drho, nc, nx, active); RTE_NOTE_LAUNCH();
    } else {
      extract_rho32_kernel<<<gv, 256, 0, st>>>(s->xl[0]->p, drho, nc, nx, active); RTE_NOTE_LAUNCH();
    }
    RTE_CUDA_TRY(cudaGetLastError());
    return RTE_OK;
  }
  if (base) return fail(RTE_EINVAL, "DSA: the fused update needs a single V-cycle");
  pack_rhs32_kernel<<<gv, 256, 0, st>>>(R, s->borig.p, nc, nx, active); RTE_NOTE_LAUNCH();
  const LevelC L0 = lvl_of(bt, 0);
  for (int it = 0; it < k; ++it) {
    if (it == 0) {
      RTE_CUDA_TRY(cudaMemcpyAsync(s->bl[0]->p, s->borig.p, sizeof(float) * (size_t)B * per,
                                   cudaMemcpyDeviceToDevice, st));
    } else {
      residual_ext_kernel<<<dim3((nc + 127) / 128, B), 128, 0, st>>>(L0, s->borig.p, s->xtot.p,
                                                                   s->bl[0]->p, active); RTE_NOTE_LAUNCH();
    }
    RTE_TRY(vcycle(bt, 0, active, st, bt->dsa_nu));
    if (it == 0) {
      RTE_CUDA_TRY(cudaMemcpyAsync(s->xtot.p, s->xl[0]->p, sizeof(float) * (size_t)B * per,
                                   cudaMemcpyDeviceToDevice, st));
    } else {
      add32_kernel<<<gvc, 256, 0, st>>>(s->xl[0]->p, s->xtot.p, (int)per, active); RTE_NOTE_LAUNCH();
    }
  }
  extract_rho32_kernel<<<gv, 256, 0, st>>>(s->xtot.p, drho, nc, nx, active); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  return RTE_OK;
}

static int dsa2d_fgmres(rte_batch_t bt, const double* R, double* drho, double rtol, int max_it,
                        const uint8_t* active_in, int* iters_out, cudaStream_t st) {
  DsaState* s = bt->dsa;
  const rte_disc_s* d = bt->disc;
  RTE_TRY(dsa_krylov_alloc(bt));
  const int B = bt->B, nc = d->n_cells, n = nc * NB, m = s->m;
  const size_t vstride = (size_t)B * n;
  const Fine F = fine_of(bt);
  // host copy of the active mask (instances drop out as they converge)
  std::vector<uint8_t> act(B, 1);
  if (active_in) RTE_CUDA_TRY(cudaMemcpy(act.data(), active_in, B, cudaMemcpyDeviceToHost));
  DevBuf<uint8_t> act_dev;
  RTE_TRY(act_dev.alloc(B));
  auto upload_act = [&]() -> int {
    RTE_CUDA_TRY(cudaMemcpyAsync(act_dev.p, act.data(), B, cudaMemcpyHostToDevice, st));
    return RTE_OK;
  };
  RTE_TRY(upload_act());
  const dim3 gvec((n + 255) / 256, B), gvec_c(std::min((n + 255) / 256, 512), B);
  double* x = s->xs.p;
  RTE_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * vstride, st));
  std::vector<double> beta0(B, 0.0), hbuf((size_t)B * (m + 1));
  std::vector<int> its(B, 0);
  std::vector<uint8_t> done(B, 0);
  for (int b = 0; b < B; ++b) done[b] = !act[b];
  int status = RTE_OK;
  // r0 = b - A x (x = 0 initially): v0 = packed R
  double* w = s->w.p;
  pack_rhs_kernel<<<gvec, 256, 0, st>>>(R, w, nc, act_dev.p); RTE_NOTE_LAUNCH();
  bool first = true;
  int total_it = 0;
  while (true) {
    // w holds the current residual for active instances
    dots_kernel<<<dim3(1, B), 512, 0, st>>>(w, 0, w, s->dots_dev.p, n, m + 1, act_dev.p); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaMemcpyAsync(hbuf.data(), s->dots_dev.p, sizeof(double) * B * (m + 1),
                                 cudaMemcpyDeviceToHost, st));
    RTE_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> beta(B, 0.0);
    for (int b = 0; b < B; ++b) {
      if (!act[b]) continue;
      beta[b] = std::sqrt(std::max(hbuf[(size_t)b * (m + 1)], 0.0));
      if (first) beta0[b] = beta[b];
      if (beta[b] <= rtol * beta0[b] || beta[b] == 0.0 || total_it >= max_it) {
        act[b] = 0;
        done[b] = 1;
        if (total_it >= max_it && beta[b] > rtol * beta0[b]) status = RTE_ENOCONV;
      }
    }
    first = false;
    bool any = false;
    for (int b = 0; b < B; ++b) any |= act[b] != 0;
    if (!any) break;
    RTE_TRY(upload_act());
    // v0 = w / beta
    std::vector<double> inv((size_t)B * (m + 1), 0.0);
    for (int b = 0; b < B; ++b) inv[(size_t)b * (m + 1)] = act[b] ? 1.0 / beta[b] : 0.0;
    RTE_CUDA_TRY(cudaMemcpyAsync(s->dots_dev.p, inv.data(), sizeof(double) * inv.size(),
                                 cudaMemcpyHostToDevice, st));
    scale_kernel<<<gvec_c, 256, 0, st>>>(w, s->V.p, s->dots_dev.p, n, m + 1, act_dev.p); RTE_NOTE_LAUNCH();
    // Arnoldi with Givens rotations per instance
    std::vector<double> H((size_t)B * (m + 1) * m, 0.0), cs((size_t)B * m), sn((size_t)B * m),
        g((size_t)B * (m + 1), 0.0);
    for (int b = 0; b < B; ++b) g[(size_t)b * (m + 1)] = beta[b];
    std::vector<uint8_t> inner(act);
    std::vector<int> kdone(B, 0);
    int k = 0;
    for (; k < m; ++k) {
      bool anyi = false;
      for (int b = 0; b < B; ++b) anyi |= inner[b] != 0;
      if (!anyi) break;
      RTE_CUDA_TRY(cudaMemcpyAsync(act_dev.p, inner.data(), B, cudaMemcpyHostToDevice, st));
      double* vk = s->V.p + (size_t)k * vstride;
      double* zk = s->Z.p + (size_t)k * vstride;
      // z_k = M^{-1} v_k (one FP32 V-cycle)
      to32_kernel<<<gvec_c, 256, 0, st>>>(vk, s->bl[0]->p, nc, d->nx, act_dev.p); RTE_NOTE_LAUNCH();
      RTE_TRY(vcycle(bt, 0, act_dev.p, st, bt->dsa_nu));
      to64_kernel<<<gvec_c, 256, 0, st>>>(s->xl[0]->p, zk, nc, d->nx, act_dev.p); RTE_NOTE_LAUNCH();
      // w = A z_k (FP64)
      fine_apply64_kernel<<<gvec, 256, 0, st>>>(F, d->nx, d->ny, B, zk, w, act_dev.p); RTE_NOTE_LAUNCH();
      // classical Gram-Schmidt, twice
      std::vector<double> hk((size_t)B * (m + 1), 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        dots_kernel<<<dim3(k + 1, B), 512, 0, st>>>(s->V.p, vstride, w, s->dots_dev.p, n, m + 1,
                                                    act_dev.p); RTE_NOTE_LAUNCH();
        gs_update_kernel<<<gvec_c, 256, 0, st>>>(s->V.p, vstride, w, s->dots_dev.p, n, k + 1,
                                                 m + 1, act_dev.p); RTE_NOTE_LAUNCH();
        RTE_CUDA_TRY(cudaMemcpyAsync(hbuf.data(), s->dots_dev.p, sizeof(double) * B * (m + 1),
                                     cudaMemcpyDeviceToHost, st));
        RTE_CUDA_TRY(cudaStreamSynchronize(st));
        for (int b = 0; b < B; ++b)
          if (inner[b])
            for (int i = 0; i <= k; ++i) hk[(size_t)b * (m + 1) + i] += hbuf[(size_t)b * (m + 1) + i];
      }
      dots_kernel<<<dim3(1, B), 512, 0, st>>>(w, 0, w, s->dots_dev.p, n, m + 1, act_dev.p); RTE_NOTE_LAUNCH();
      RTE_CUDA_TRY(cudaMemcpyAsync(hbuf.data(), s->dots_dev.p, sizeof(double) * B * (m + 1),
                                   cudaMemcpyDeviceToHost, st));
      RTE_CUDA_TRY(cudaStreamSynchronize(st));
      std::vector<double> sc((size_t)B * (m + 1), 0.0);
      ++total_it;
      for (int b = 0; b < B; ++b) {
        if (!inner[b]) continue;
        double* hcol = &hk[(size_t)b * (m + 1)];
        hcol[k + 1] = std::sqrt(std::max(hbuf[(size_t)b * (m + 1)], 0.0));
        sc[(size_t)b * (m + 1)] = hcol[k + 1] > 0 ? 1.0 / hcol[k + 1] : 0.0;
        // apply previous rotations
        for (int i = 0; i < k; ++i) {
          const double c = cs[(size_t)b * m + i], sn_ = sn[(size_t)b * m + i];
          const double t = c * hcol[i] + sn_ * hcol[i + 1];
          hcol[i + 1] = -sn_ * hcol[i] + c * hcol[i + 1];
          hcol[i] = t;
        }
        const double den = std::hypot(hcol[k], hcol[k + 1]);
        const double c = den > 0 ? hcol[k] / den : 1.0, sn_ = den > 0 ? hcol[k + 1] / den : 0.0;
        cs[(size_t)b * m + k] = c, sn[(size_t)b * m + k] = sn_;
        hcol[k] = den;
        hcol[k + 1] = 0.0;
        double* gb = &g[(size_t)b * (m + 1)];
        gb[k + 1] = -sn_ * gb[k];
        gb[k] = c * gb[k];
        for (int i = 0; i <= k; ++i) H[((size_t)b * (m + 1) + i) * m + k] = hcol[i];
        kdone[b] = k + 1;
        its[b] += 1;
        if (std::fabs(gb[k + 1]) <= rtol * beta0[b] || total_it >= max_it) inner[b] = 0;
      }
      // v_{k+1} = w / h_{k+1,k}
      if (k + 1 <= m) {
        RTE_CUDA_TRY(cudaMemcpyAsync(s->dots_dev.p, sc.data(), sizeof(double) * sc.size(),
                                     cudaMemcpyHostToDevice, st));
        scale_kernel<<<gvec_c, 256, 0, st>>>(w, s->V.p + (size_t)(k + 1) * vstride, s->dots_dev.p, n,
                                             m + 1, act_dev.p); RTE_NOTE_LAUNCH();
      }
    }
    // solve H y = g and update x += Z y
    std::vector<double> y((size_t)B * (m + 1), 0.0);
    int kmax = 0;
    for (int b = 0; b < B; ++b) {
      if (!act[b]) continue;
      const int kb = kdone[b];
      kmax = std::max(kmax, kb);
      for (int i = kb - 1; i >= 0; --i) {
        double sacc = g[(size_t)b * (m + 1) + i];
        for (int j2 = i + 1; j2 < kb; ++j2) sacc -= H[((size_t)b * (m + 1) + i) * m + j2] * y[(size_t)b * (m + 1) + j2];
        y[(size_t)b * (m + 1) + i] = sacc / H[((size_t)b * (m + 1) + i) * m + i];
      }
    }
    RTE_TRY(upload_act());
    RTE_CUDA_TRY(cudaMemcpyAsync(s->dots_dev.p, y.data(), sizeof(double) * y.size(),
                                 cudaMemcpyHostToDevice, st));
    combine_kernel<<<gvec_c, 256, 0, st>>>(s->Z.p, vstride, x, s->dots_dev.p, n, kmax, m + 1,
                                           act_dev.p); RTE_NOTE_LAUNCH();
    // new residual w = b - A x
    fine_apply64_kernel<<<gvec, 256, 0, st>>>(F, d->nx, d->ny, B, x, w, act_dev.p); RTE_NOTE_LAUNCH();
    {
      // w = packed(R) - w  (reuse V_m as scratch for the packed right-hand side)
      double* pr = s->V.p + (size_t)m * vstride;
      pack_rhs_kernel<<<gvec, 256, 0, st>>>(R, pr, nc, act_dev.p); RTE_NOTE_LAUNCH();
      std::vector<double> mone((size_t)B * (m + 1), 0.0);
      for (int b = 0; b < B; ++b) mone[(size_t)b * (m + 1)] = 1.0;
      RTE_CUDA_TRY(cudaMemcpyAsync(s->dots_dev.p, mone.data(), sizeof(double) * mone.size(),
                                   cudaMemcpyHostToDevice, st));
      // w <- w - 1 * pr, then negate via scale by -1
      gs_update_kernel<<<gvec_c, 256, 0, st>>>(pr, 0, w, s->dots_dev.p, n, 1, m + 1, act_dev.p); RTE_NOTE_LAUNCH();
      for (int b = 0; b < B; ++b) mone[(size_t)b * (m + 1)] = -1.0;
      RTE_CUDA_TRY(cudaMemcpyAsync(s->dots_dev.p, mone.data(), sizeof(double) * mone.size(),
                                   cudaMemcpyHostToDevice, st));
      scale_kernel<<<gvec_c, 256, 0, st>>>(w, w, s->dots_dev.p, n, m + 1, act_dev.p); RTE_NOTE_LAUNCH();
    }
    RTE_CUDA_TRY(cudaGetLastError());
    if (total_it >= max_it) {
      // final convergence check happens at the top of the loop
    }
  }
  // drho = rho-field of x for the instances that were requested
  std::vector<uint8_t> req(B, 1);
  if (active_in) RTE_CUDA_TRY(cudaMemcpy(req.data(), active_in, B, cudaMemcpyDeviceToHost));
  RTE_CUDA_TRY(cudaMemcpyAsync(act_dev.p, req.data(), B, cudaMemcpyHostToDevice, st));
  extract_rho_kernel<<<dim3((nc * 4 + 255) / 256, B), 256, 0, st>>>(x, drho, nc, act_dev.p); RTE_NOTE_LAUNCH();
  RTE_CUDA_TRY(cudaGetLastError());
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  if (iters_out)
    for (int b = 0; b < B; ++b) iters_out[b] = its[b];
  return status;
}

bool dsa_update_fusable(rte_batch_t bt, double rtol, int max_it) {
  return bt->dsa && bt->disc->dim == 2 && rtol == 0.0 && max_it == 1;
}

int dsa_apply_update(rte_batch_t bt, const double* R, const double* rho_star, double* rho_out,
                     const uint8_t* active, cudaStream_t st) {
  if (!dsa_update_fusable(bt, 0.0, 1)) return fail(RTE_EINVAL, "DSA: fused update not available");
  return dsa2d_vcycles(bt, R, rho_out, 1, active, st, rho_star);
}

int dsa_apply(rte_batch_t bt, const double* R, double* drho, double rtol, int max_it,
              const uint8_t* active, int* iters, cudaStream_t st) {
  DsaState* s = bt->dsa;
  if (!s) return fail(RTE_ESTATE, "DSA not set up");
  if (bt->disc->dim == 1) {
    dsa1d_solve_kernel<<<(bt->B + 63) / 64, 64, 0, st>>>(s->K1, s->Dpinv.p, s->Mfac.p, R, drho,
                                                         s->work1.p, bt->disc->nx, bt->B, active); RTE_NOTE_LAUNCH();
    RTE_CUDA_TRY(cudaGetLastError());
    if (iters)
      for (int b = 0; b < bt->B; ++b) iters[b] = 1;
    return RTE_OK;
  }
  if (rtol == 0.0) {  // fixed number of V-cycles, no synchronisation
    RTE_TRY(dsa2d_vcycles(bt, R, drho, max_it, active, st));
    if (iters)
      for (int b = 0; b < bt->B; ++b) iters[b] = max_it;
    return RTE_OK;
  }
  return dsa2d_fgmres(bt, R, drho, rtol, max_it, active, iters, st);
}

}  // namespace rte

using namespace rte;

extern "C" int rte_dsa_correction(rte_batch_t b, const double* R, double* drho, double rtol,
                                  int max_it, const uint8_t* active, int* iters, void* stream) {
  if (!b || !R || !drho) return fail(RTE_EINVAL, "rte_dsa_correction: null argument");
  RTE_TRY(params_ready(b, "rte_dsa_correction"));
  if (!(rtol >= 0) || max_it < 1) return fail(RTE_EINVAL, "rte_dsa_correction: bad tolerance");
  DeviceGuard g(b->disc->device);
  cudaStream_t st = (cudaStream_t)stream;
  int s = dsa_apply(b, R, drho, rtol, max_it, active, iters, st);
  if (s != RTE_OK && s != RTE_ENOCONV) return s;
  RTE_CUDA_TRY(cudaStreamSynchronize(st));
  return s;
}

extern "C" int rte_batch_dsa_smoother(rte_batch_t b, int kind) {
  if (!b || kind < RTE_SMOOTHER_GLOBAL || kind > RTE_SMOOTHER_BLOCKED)
    return fail(RTE_EINVAL, "rte_batch_dsa_smoother: unknown smoother");
  b->dsa_tiled = kind == RTE_SMOOTHER_TILED;
  b->dsa_blocking = kind == RTE_SMOOTHER_BLOCKED;
  return RTE_OK;
}

extern "C" int rte_batch_dsa_smoothing(rte_batch_t b, int nu) {
  if (!b || nu < 1 || nu > 8) return fail(RTE_EINVAL, "rte_batch_dsa_smoothing: need 1 <= nu <= 8");
  b->dsa_nu = nu;
  return RTE_OK;
}
