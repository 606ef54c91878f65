// Host stand-in for the cluster API of cooperative groups, as the library's block solve uses it:
// a cluster of one CTA (one block, rank 0, its own shared memory, a barrier that has nothing to
// wait for). Only the per-pair math of that header is run on the host; nothing here runs on a GPU.
#pragma once
namespace cooperative_groups {
struct host_cluster {
  void sync() const {}
  unsigned num_blocks() const { return 1; }
  unsigned block_rank() const { return 0; }
  template <class T>
  T* map_shared_rank(T* p, unsigned) const { return p; }
};
inline host_cluster this_cluster() { return {}; }
}  // namespace cooperative_groups
