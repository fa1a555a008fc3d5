// Host-side helpers shared by the C ABI translation units (internal).
#pragma once

#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lcbp {

// parameters of one lattice / replica, in double on the host
struct HostParams {
  double A0, gamma, K, q0;  // Landau-de Gennes (Sec. 2.1 Eq. free_energy)
  double tau_f, xi, Gamma;  // kinetics (Sec. 2.1, 2.2)
  int flow_on, coupling;
  int walls_z;              // solid walls below z = 0 and above z = nz-1
  double q_wall[5];         // anchored Q beyond the walls (q5 order)
  int l2_set;               // 0: one-constant energy (L2 = K); 1: L2 below
  double L2;
  double rho0;              // reference density (initial f^eq when no density is given)
};

extern thread_local std::string g_last_error;
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

TileShape default_tile(int nx, int ny, int nz);
long long tile_count(int nx, int ny, int nz, TileShape t);
void append_tiles(std::vector<Tile>& out, int rep, int nx, int ny, int nz, TileShape t);
bool valid_dtype(int d);
size_t dtype_size(int d);
size_t replica_bytes(int dtype);
template <typename real>
void fill_replica(void* dst, int nx, int ny, int nz, long long base, const HostParams& p);
double s_eq(double gamma);
int check_params(const HostParams& p);
int transfer(void* state, int sd, void* user, int ud, long long count, bool upload, void* staging,
             long long staging_elems, cudaStream_t st);
bool encode_tiled(CUtensorMap* tm, void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                  const cuuint32_t* box, int dtype);

}  // namespace lcbp
