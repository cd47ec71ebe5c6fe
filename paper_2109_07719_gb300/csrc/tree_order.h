// Link order of one system for the batched kernels: depth-first preorder, the
// children of a link visited in ascending order of the model's numbering.  In
// this order a link's subtree is a contiguous range, a link with children has
// link l + 1 as its first child, and the values a branching link hands to (or
// collects from) its later children nest: the world-aligned passes keep them on a
// stack whose depth is the nesting of branchings along a path, not the link count.
// Host code only; shared by the library's model packing and the host checks.
#pragma once

#include <algorithm>
#include <vector>

namespace abasim {

struct TreeOrder {
  std::vector<int> perm;     // stored position -> the model's link index
  std::vector<int> pos;      // the model's link index -> stored position
  std::vector<int> parent;   // parent of each stored position (-1: the world)
  std::vector<char> branch;  // the link has a child other than link l + 1 (several children)
  std::vector<char> lastsib; // the last child of a branching link (never its first, link parent + 1)
  int depth = 0;             // the most stack entries a pass holds at once
};

// parent[l] < l for every link (-1: attached to the world), n links.
inline TreeOrder tree_order(const int* parent, int n) {
  TreeOrder t;
  t.pos.assign(n, 0);
  std::vector<std::vector<int>> kids(n);
  std::vector<int> todo;
  for (int l = n - 1; l >= 0; --l) {  // children lists (and the roots) in descending order
    if (parent[l] >= 0)
      kids[parent[l]].push_back(l);
    else
      todo.push_back(l);
  }
  while (!todo.empty()) {  // the smallest pending link is at the back
    const int l = todo.back();
    todo.pop_back();
    t.pos[l] = (int)t.perm.size();
    t.perm.push_back(l);
    for (int c : kids[l]) todo.push_back(c);
  }
  t.parent.assign(n, -1);
  std::vector<int> nkids(n, 0), lastkid(n, -1);
  for (int l = 0; l < n; ++l) {
    const int p = parent[t.perm[l]];
    t.parent[l] = p >= 0 ? t.pos[p] : -1;
    if (t.parent[l] >= 0) {
      ++nkids[t.parent[l]];
      lastkid[t.parent[l]] = std::max(lastkid[t.parent[l]], l);
    }
  }
  t.branch.assign(n, 0);
  t.lastsib.assign(n, 0);
  int sp = 0;
  for (int l = 0; l < n; ++l) {  // the outward passes' stack; the inward ones mirror it
    const int p = t.parent[l];
    t.branch[l] = nkids[l] > 1;
    t.lastsib[l] = p >= 0 && p != l - 1 && lastkid[p] == l;
    if (t.lastsib[l]) --sp;
    if (t.branch[l]) t.depth = std::max(t.depth, ++sp);
  }
  return t;
}

}  // namespace abasim
