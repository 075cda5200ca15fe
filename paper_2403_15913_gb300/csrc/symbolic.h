// Host-side symbolic analysis of the condensed KKT matrix (Sec. V-B of
// Pacaud & Shin: the pattern of K is fixed across IPM iterations, so the
// ordering and symbolic factorisation are computed once and reused by every
// refactorisation).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace kktgb {

struct SymbolicOptions {
    int leaf_size = 64;
    int relax_cols = 48;
    int relax_zeros = 1024;
    int max_width = 64;
    bool parallel = true;   // fork the top of the nested-dissection recursion
                            // onto threads (the result does not depend on it)
};

// Result of the analysis.  All column/row labels after `perm` are in the
// permuted ("new") numbering of P K P^T.
struct Symbolic {
    int n = 0;
    std::vector<int> perm;      // new -> old
    std::vector<int> iperm;     // old -> new
    std::vector<int> parent;    // elimination tree, -1 for roots
    std::vector<int> colcount;  // nnz of every column of L (diagonal included)
    std::vector<int> sn_ptr;    // supernode column boundaries (ns + 1)
    std::vector<int> sn_rowptr; // offsets into sn_rows (ns + 1)
    std::vector<int> sn_rows;   // rows(s), ascending, starting with cols(s)
    std::vector<int> sn_parent; // supernodal tree, -1 for roots
    // For every entry q of sn_rows (row i of supernode s): bit k is set when
    // L(i, first(s) + k) is structurally nonzero (true structure, not the
    // explicit zeros of relaxed panels).  Filled only when every supernode
    // has at most 64 columns (otherwise empty).
    std::vector<uint64_t> sn_rowmask;
    double flops = 0.0;         // sum_j colcount_j^2
    int64_t nnz_L = 0;
    int ns() const { return (int)sn_ptr.size() - 1; }
};

// Undirected graph of pattern(W + J^T J) without self loops, CSR with
// sorted, duplicate-free adjacency lists.
struct Graph {
    int n = 0;
    std::vector<int64_t> xadj;
    std::vector<int> adj;
};

// Returns an empty string on success, otherwise a message.
std::string build_graph(int n, int m, const int* W_colptr, const int* W_rowind,
                        const int* J_rowptr, const int* J_colind, Graph& g);
std::string analyse(const Graph& g, const SymbolicOptions& opt, Symbolic& out);

// Analysis of a block-diagonal union from the analyses of its blocks, in
// block order: labels, supernodes and row lists are offset and appended.
// Equal to analysing the union's pattern, because the ordering takes
// connected components in the order of their smallest vertex and every later
// step (elimination tree, postorder with roots in increasing order, column
// counts, supernodes, relaxation along tree edges, row lists) is local to
// the elimination tree of one block.
void concat(const std::vector<Symbolic>& parts, Symbolic& out);

}  // namespace kktgb
