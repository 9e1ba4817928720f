// Persistent batch kernel (batch_team.cu): one cooperative launch runs every FP32
// instance of a batch, small ones whole in one CTA, larger ones on teams of CTAs.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace cheb {

// One instance of the batch (device descriptor; the slots of an instance are
// [first_slot, first_slot + max(team, 1))).
struct TeamInst {
    int n, K, Q;
    int team;        // 0: whole run in one CTA's shared memory (n <= 13); else CTAs of the team
    int l, H;        // low-pass partner bits in L2 and strided bits (team_split)
    int first_slot;
    int pad;
    double g;        // gamma / r
    const double2* coef;    // c_0..c_K, device
    const int64_t* tiles;   // energy tables (11-bit tiles), device
    const int64_t* elow;
    float4* psi;            // the state (two complex64 per float4), in/out
    float4* v0;             // Clenshaw vectors (workspace)
    float4* v1;
    unsigned* bar;          // team barrier counter, zero at launch
};

// CTAs of the team of an n-qubit instance (0 for the whole-run kernel), for a launch of
// ctas_per_sm CTAs per SM.
int team_size(int n, int ctas_per_sm);
// Split of the flips: l low-pass partner bits in L2, H bits in one strided pass.
void team_split(int n, int* l, int* H);
// ctas_per_sm: 1 (128 registers per thread, the default) or 2 (64 registers).
cudaError_t launch_batch_team(const TeamInst* inst, int ninst, int nslots, unsigned* slot_counter, int* flags,
                              int ctas_per_sm, cudaStream_t s);

// Failure-detection self-test of the team barrier: one CTA of a team of two waits, with
// `limit` clock cycles, for a teammate that never arrives (bar must be zero).
cudaError_t launch_team_barrier_selftest(unsigned* bar, int* flags, long long limit, cudaStream_t s);

}  // namespace cheb
