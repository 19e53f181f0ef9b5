// molt_recv.cuh -- receivers: traces of a time level at given nodes, and the
// injection of receiver values into a level (the sources of the adjoint
// recursion).  Shared by the single-problem and the batched entry points;
// a node is an index into the level's own layout.
#pragma once
#include <algorithm>
#include <vector>

namespace molt {

// out[r] = level value at irec[r]
template <class T>
__global__ void k_recv_gather(const T *hi, const T *lo, const long long *irec, int nrec, double *out)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x) {
        const long long i = irec[r];
        double v = (double)hi[i];
        if constexpr (sizeof(T) == 4) v += (double)lo[i];
        out[r] = v;
    }
}

// level[node[u]] += the values of the node's receivers, added in receiver
// order (order[start[u]] .. order[start[u+1] - 1]); one thread per distinct
// node, so receivers that share a node need no atomics and the sum is the
// same on every run
template <class T>
__global__ void k_recv_inject(T *hi, T *lo, const long long *node, const long long *start, const long long *order,
                              int nnode, const double *vals)
{
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nnode; u += gridDim.x * blockDim.x) {
        const long long i = node[u];
        double x = (double)hi[i];
        if constexpr (sizeof(T) == 4) x += (double)lo[i];
        for (long long j = start[u]; j < start[u + 1]; ++j) x += vals[order[j]];
        if constexpr (sizeof(T) == 4) {
            const float h = __double2float_rn(x);
            hi[i] = h;
            lo[i] = __double2float_rn(x - (double)h);
        } else {
            hi[i] = x;
        }
    }
}

// Host layout of the receiver buffer (4 nrec + 1 entries): the receivers'
// nodes in receiver order, then the distinct nodes (nnode of nrec slots),
// the groups' starts (nrec + 1 slots) and the receivers grouped by node
// (stable: each group in receiver order).  Returns nnode.
inline int receiver_layout(const std::vector<long long> &ir, std::vector<long long> &buf)
{
    const int nrec = (int)ir.size();
    std::vector<int> ord(nrec);
    for (int r = 0; r < nrec; ++r) ord[r] = r;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return ir[x] < ir[y]; });
    buf.assign(4 * (size_t)nrec + 1, 0);
    long long *node = buf.data() + nrec, *start = node + nrec, *order = start + nrec + 1;
    int nn = 0;
    for (int j = 0; j < nrec; ++j) {
        if (j == 0 || ir[ord[j]] != ir[ord[j - 1]]) {
            node[nn] = ir[ord[j]];
            start[nn++] = j;
        }
        order[j] = ord[j];
    }
    start[nn] = nrec;
    for (int r = 0; r < nrec; ++r) buf[r] = ir[r];
    return nn;
}

}  // namespace molt
