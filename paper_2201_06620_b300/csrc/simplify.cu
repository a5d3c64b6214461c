// rosnet_simplify: rank reduction of a tensor network before path search.
//
// The paper builds and simplifies its circuit networks with a front end
// before the contraction path is chosen (Sec. V): tensors of rank 1 and 2
// (initial states, one-qubit gates, output projectors) are absorbed into a
// neighbour, which leaves a network of about one tensor per two-qubit gate.
// Here the choice of merges is host logic and every merge is one pairwise
// tensordot on the device (rosnet_tensordot), so the merged tensors are
// computed by the library's kernels like any other step.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <vector>

#include "internal.h"

namespace rosnet {
namespace {

struct Node {
    rosnet_btensor t = nullptr;
    std::vector<int64_t> labels;
    bool alive = true;
    bool keep = false;
    bool created = false;   // made by this call (freed if absorbed in turn)
};

}  // namespace
}  // namespace rosnet

extern "C" rosnet_status rosnet_simplify(const rosnet_network *net, const uint8_t *keep, int32_t max_rank,
                                         const rosnet_opts *opts, void *stream, rosnet_btensor *tensors_out,
                                         int32_t *ranks_out, int64_t *labels_out, int32_t *origin_out,
                                         int32_t *ntensors_out) {
    using namespace rosnet;
    if (!net || !tensors_out || !ranks_out || !origin_out || !ntensors_out || max_rank < 0 || max_rank > 2)
        return ROSNET_ERR_INVALID_ARG;
    if (net->ntensors < 0 || (net->ntensors > 0 && (!net->tensors || !net->ranks || !net->labels)) ||
        net->nout < 0 || (net->nout > 0 && !net->out_labels))
        return ROSNET_ERR_INVALID_ARG;
    RN_API_BEGIN
    const int n = net->ntensors;
    std::vector<Node> nodes(n);
    size_t total_labels = 0;
    std::map<int64_t, int> count;   // tensors carrying each label
    for (int i = 0; i < n; ++i) {
        rosnet_btensor t = net->tensors[i];
        if (!t) RN_FAIL(ROSNET_ERR_INVALID_ARG, "null tensor in the network");
        if (net->ranks[i] != t->lay.rank) RN_FAIL(ROSNET_ERR_INVALID_ARG, "rank does not match the tensor");
        if (net->ranks[i] > 0 && !net->labels[i]) RN_FAIL(ROSNET_ERR_INVALID_ARG, "labels are NULL");
        nodes[i].t = t;
        nodes[i].labels.assign(net->labels[i], net->labels[i] + net->ranks[i]);
        nodes[i].keep = keep && keep[i];
        total_labels += net->ranks[i];
        for (int64_t l : nodes[i].labels) ++count[l];
    }
    if (total_labels > 0 && !labels_out) RN_FAIL(ROSNET_ERR_INVALID_ARG, "labels_out is NULL");
    for (int i = 0; i < net->nout; ++i) count[net->out_labels[i]] += 2;   // never summed
    try {
        bool changed = true;
        while (changed) {
            changed = false;
            for (int i = 0; i < n; ++i) {
                Node &a = nodes[i];
                if (!a.alive || a.keep || (int)a.labels.size() > max_rank) continue;
                // the neighbour: not kept, sharing only labels carried by these
                // two tensors alone; highest rank first, then lowest index
                int best = -1;
                for (int j = 0; j < n; ++j) {
                    const Node &b = nodes[j];
                    if (j == i || !b.alive || b.keep) continue;
                    int shared = 0;
                    bool ok = true;
                    for (int64_t l : a.labels)
                        if (std::find(b.labels.begin(), b.labels.end(), l) != b.labels.end()) {
                            ++shared;
                            ok = ok && count[l] == 2;
                        }
                    if (shared == 0 || !ok) continue;
                    if (best < 0 || b.labels.size() > nodes[best].labels.size()) best = j;
                }
                if (best < 0) continue;
                Node &b = nodes[best];
                // C = tensordot(b, a) over the shared labels: b's free labels,
                // then a's
                std::vector<int> ax_b, ax_a;
                std::vector<int64_t> lc;
                for (size_t x = 0; x < b.labels.size(); ++x) {
                    auto it = std::find(a.labels.begin(), a.labels.end(), b.labels[x]);
                    if (it != a.labels.end()) {
                        ax_b.push_back((int)x);
                        ax_a.push_back((int)(it - a.labels.begin()));
                    } else {
                        lc.push_back(b.labels[x]);
                    }
                }
                for (int64_t l : a.labels)
                    if (std::find(b.labels.begin(), b.labels.end(), l) == b.labels.end()) lc.push_back(l);
                rosnet_btensor c = nullptr;
                const rosnet_status st =
                    rosnet_tensordot(b.t, a.t, (int)ax_b.size(), ax_b.data(), ax_a.data(), opts, stream, &c);
                if (st != ROSNET_OK) RN_FAIL(st, "merge failed: " + std::string(rosnet_last_error()));
                for (int64_t l : a.labels)
                    if (std::find(b.labels.begin(), b.labels.end(), l) != b.labels.end()) count[l] -= 2;
                if (a.created) free_tensor(a.t);
                if (b.created) free_tensor(b.t);
                b.t = c;
                b.created = true;
                b.labels = lc;
                a.alive = false;
                a.t = nullptr;
                changed = true;
            }
        }
    } catch (...) {
        for (Node &x : nodes)
            if (x.created && x.t) free_tensor(x.t);
        throw;
    }
    int k = 0;
    size_t lo = 0;
    for (int i = 0; i < n; ++i) {
        if (!nodes[i].alive) continue;
        tensors_out[k] = nodes[i].t;
        ranks_out[k] = (int32_t)nodes[i].labels.size();
        origin_out[k] = i;
        for (int64_t l : nodes[i].labels) labels_out[lo++] = l;
        ++k;
    }
    *ntensors_out = k;
    return ROSNET_OK;
    RN_API_END
}
