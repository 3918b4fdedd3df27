// Internal structures of libsie (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sie.h"

struct sie_mesh {
    std::vector<double> xyz;      // [nv][3]
    std::vector<int32_t> tri;     // [nt][3]
    std::vector<int32_t> cond;    // [nt]
    std::vector<double> sigma;    // [ncond]
    int64_t nv = 0, nt = 0;
    int32_t ncond = 0;
};

// Circuit graph and fundamental loops (Sec. II-D, III).
struct sie_loops {
    int64_t nt = 0, n_nodes = 0, nb = 0, n_comp = 0, nl = 0, np = 0, depth = 0;
    std::vector<int64_t> node_of_tri;            // [nt]
    std::vector<int32_t> br_tri;                 // [nb][2]  T+, T-
    std::vector<int8_t> br_local;                // [nb][2]  local edge (opposite vertex)
    std::vector<int32_t> tail, head;             // [nb + np]
    std::vector<int32_t> parent, parent_branch;  // [n_nodes]
    std::vector<int32_t> comp;                   // [n_nodes]
    std::vector<int32_t> link_branch;            // [nl]
    std::vector<int32_t> loop_of_branch;         // [nb + np], -1 for twigs
    std::vector<int32_t> port_src, port_sink;    // [np] nodes
    // loop matrix A, CSR over loops, columns in walk order
    std::vector<int64_t> a_ptr;
    std::vector<int32_t> a_col;
    std::vector<int8_t> a_val;
    // Euler tour of the spanning forest: 2 n_nodes slots
    std::vector<int32_t> enter, exit_;           // [n_nodes] tour positions
    std::vector<int32_t> tour_node;              // [2 n_nodes] node at slot
    std::vector<int8_t> tour_is_enter;           // [2 n_nodes]
    // per node: incident links as (loop id, +1 if the link enters the node)
    std::vector<int32_t> nl_ptr, nl_loop;
    std::vector<int8_t> nl_sign;
};

namespace sie {
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
}  // namespace sie
