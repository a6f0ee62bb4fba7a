// Internal C++ interface of the shared-round executor (randrand.cu) for the
// serving loop (server.cu).  Not part of the C ABI.
#pragma once
#include <vector>

#include "rr_common.cuh"

struct rr_handle;

namespace rr {

struct Group;   // opaque: a GroupExec of randrand.cu

// one system handed to the rounds: a built handle and its solve request;
// `user` comes back with the outcome
struct GroupReq {
  rr_handle* h;
  const double* b;
  double* x;
  int64_t ldb, ldx;
  int m;
  double rtol;
  int maxit;
  rr_solve_info* info;   // m entries, written when the system finishes
  void* user;
};
struct GroupDone {
  void* user;
  rr_status status;
};

// the handle can iterate in the rounds of a group with mp columns and k <= kmax
bool group_accepts(const rr_handle* h, int mp, int kmax);
// device bytes of a group with this capacity; part_bytes: its partial-sum pool
size_t group_bytes(int mp, int maxsys, int64_t max_rows, size_t part_bytes);
Group* group_create(int mp, int kmax, int maxsys, int64_t max_rows, size_t part_bytes, void* ws,
                    size_t ws_bytes, cudaStream_t st, rr_status* s);
// join: RR_OK (in the rounds, or already finished: then `done` holds it),
// RR_ERR_WORKSPACE when the group is full now (retry after systems leave),
// another status when the system cannot run in the rounds (not joined)
rr_status group_add(Group* g, const GroupReq& r, std::vector<GroupDone>* done);
// one replay of the rounds and the restarts after it; finished systems are
// appended to `done` (their handles are back on their own streams)
rr_status group_step(Group* g, std::vector<GroupDone>* done);
int group_size(const Group* g);
// host wall-clock split of the replay loop so far (rr_rounds_stats)
void group_stats(const Group* g, rr_rounds_stats* out);
void group_destroy(Group* g);

}  // namespace rr
