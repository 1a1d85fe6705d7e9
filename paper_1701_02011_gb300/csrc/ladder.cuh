// Density-fitted particle-particle ladder core shared by the energy driver
// and the standalone C entry points.
#pragma once
#include <string>

#include "engine.cuh"

namespace dsrg {

// L[p,q,i,j] += sum_{r,s} (sum_Q B[Q,p0+p,p0+r] B[Q,p0+q,p0+s]) t[r,s,i,j]
// for p,q,r,s in [0,np), i,j in [0,nh).  B is [naux][n][n] (row-major), t is
// addressed with strides tst[0..3], L is contiguous [np][np][nh][nh].  The
// (pr|qs) rows are built bp at a time into G (capacity bp * np^3 doubles).
// Launches go through `ws` (counted, optionally timed) when it is non-null.
void ladder_core(const double* B, long long n, int naux, int p0, int np, int nh, const double* t,
                 const long long* tst, double* L, double* G, long long bp, cudaStream_t st, Workspace* ws);
// The same sum for a t with t[r,s,i,j] = t[s,r,j,i] (L must be zero on
// entry), using (pr|qs) = (qs|pr): about half the work; G holds at most
// max_doubles doubles.
void ladder_core_sym(const double* B, long long n, int naux, int p0, int np, int nh, const double* t,
                     const long long* tst, double* L, double* G, long long max_doubles, cudaStream_t st,
                     Workspace* ws);
// Largest batch of p rows whose (pr|qs) fits in max_doubles (0 if none).
long long ladder_batch_rows(int np, long long max_doubles);
int ladder_check_args(int n, int naux, int p0, int np, int nh, const void* B, const void* t, const void* L,
                      std::string& msg);

// sets the calling thread's dsrg_last_error message and returns code
int set_error(int code, const char* msg);

}  // namespace dsrg
