// Host side of libsie: error state, mesh loading and the loop basis.
//
// Loop basis (Sec. II-D, Sec. III of arXiv 2210.04891): triangles are circuit
// nodes, edges shared by two triangles are branches oriented from the lower to
// the higher triangle index (the modified RWG current flows T+ -> T-).  The
// contact faces of each port are contracted into one node.  A breadth-first
// spanning forest (root = lowest node id of each part, neighbours in ascending
// branch id) splits the branches into twigs and links; each link closes one
// fundamental loop.  Port p adds a link from its sink node to its source node;
// port loops come last.  Besides the explicit loop matrix A (exported for
// checks), the forest's Euler tour is kept: A^T x and A y are then evaluated on
// the device as prefix sums along the tour (subtree sums and root-path sums),
// O(nodes) work instead of O(sum of loop lengths).
#include <algorithm>
#include <charconv>
#include <cmath>
#include <cstring>
#include <deque>
#include <fstream>
#include <sstream>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "sie_internal.h"

namespace sie {
static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}
}  // namespace sie

extern "C" const char *sie_last_error(void) { return sie::g_err.c_str(); }

extern "C" int sie_mesh_load(const double *xyz, int64_t nv, const int32_t *tri, int64_t nt,
                             const int32_t *cond_id, const double *sigma, int32_t ncond,
                             sie_mesh **out) {
    if (!out) return sie::fail(SIE_ERR_ARG, "sie_mesh_load: out is NULL");
    *out = nullptr;
    if (!xyz || !tri || !cond_id || !sigma || nv < 3 || nt < 1 || ncond < 1)
        return sie::fail(SIE_ERR_ARG, "sie_mesh_load: empty or NULL input");
    if (nt > (int64_t(1) << 30) || nv > (int64_t(1) << 30))
        return sie::fail(SIE_ERR_ARG, "sie_mesh_load: mesh larger than 2^30 elements");
    for (int32_t c = 0; c < ncond; ++c)
        if (!(sigma[c] > 0.0) || !std::isfinite(sigma[c]))
            return sie::fail(SIE_ERR_ARG, "sie_mesh_load: conductivity must be positive");
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(xyz[i])) return sie::fail(SIE_ERR_ARG, "sie_mesh_load: non-finite vertex");
    for (int64_t t = 0; t < nt; ++t) {
        for (int k = 0; k < 3; ++k)
            if (tri[3 * t + k] < 0 || tri[3 * t + k] >= nv)
                return sie::fail(SIE_ERR_ARG, "sie_mesh_load: vertex index out of range");
        if (cond_id[t] < 0 || cond_id[t] >= ncond)
            return sie::fail(SIE_ERR_ARG, "sie_mesh_load: conductor id out of range");
        const double *a = xyz + 3 * tri[3 * t], *b = xyz + 3 * tri[3 * t + 1], *c = xyz + 3 * tri[3 * t + 2];
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n0 = u[1] * v[2] - u[2] * v[1], n1 = u[2] * v[0] - u[0] * v[2], n2 = u[0] * v[1] - u[1] * v[0];
        double l2 = (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(n0 * n0 + n1 * n1 + n2 * n2 > 1e-24 * l2))
            return sie::fail(SIE_ERR_ARG, "sie_mesh_load: degenerate triangle " + std::to_string(t));
    }
    sie_mesh *m = new (std::nothrow) sie_mesh;
    if (!m) return sie::fail(SIE_ERR_OOM, "sie_mesh_load: out of host memory");
    m->xyz.assign(xyz, xyz + 3 * nv);
    m->tri.assign(tri, tri + 3 * nt);
    m->cond.assign(cond_id, cond_id + nt);
    m->sigma.assign(sigma, sigma + ncond);
    m->nv = nv;
    m->nt = nt;
    m->ncond = ncond;
    *out = m;
    return SIE_OK;
}

extern "C" void sie_mesh_destroy(sie_mesh *m) { delete m; }

namespace {

// Whitespace-separated tokens of a mesh file, '#' comments skipped; numbers are
// parsed with std::from_chars (independent of the C locale).
struct MeshTokens {
    std::string text;
    size_t pos = 0;
    bool next(std::string_view &tok) {
        for (;;) {
            while (pos < text.size() && std::isspace(static_cast<unsigned char>(text[pos]))) ++pos;
            if (pos < text.size() && text[pos] == '#') {
                while (pos < text.size() && text[pos] != '\n') ++pos;
                continue;
            }
            break;
        }
        if (pos >= text.size()) return false;
        const size_t b = pos;
        while (pos < text.size() && !std::isspace(static_cast<unsigned char>(text[pos])) && text[pos] != '#') ++pos;
        tok = std::string_view(text).substr(b, pos - b);
        return true;
    }
    template <typename T> bool number(T &v) {
        std::string_view t;
        if (!next(t)) return false;
        const char *e = t.data() + t.size();
        auto r = std::from_chars(t.data(), e, v);
        return r.ec == std::errc() && r.ptr == e;
    }
};

}  // namespace

extern "C" int sie_mesh_load_file(const char *path, sie_mesh **out) {
    if (!out) return sie::fail(SIE_ERR_ARG, "sie_mesh_load_file: out is NULL");
    *out = nullptr;
    if (!path) return sie::fail(SIE_ERR_ARG, "sie_mesh_load_file: path is NULL");
    std::ifstream f(path, std::ios::binary);
    if (!f) return sie::fail(SIE_ERR_ARG, std::string("sie_mesh_load_file: cannot open ") + path);
    MeshTokens tk;
    {
        std::ostringstream ss;
        ss << f.rdbuf();
        tk.text = ss.str();
    }
    auto bad = [&](const std::string &what) {
        return sie::fail(SIE_ERR_ARG, std::string("sie_mesh_load_file: ") + path + ": " + what);
    };
    std::string_view magic;
    int version = 0;
    if (!tk.next(magic) || magic != "sie_mesh" || !tk.number(version)) return bad("not a sie_mesh file");
    if (version != 1) return bad("unsupported version " + std::to_string(version));
    int64_t nv = 0, nt = 0, nc = 0;
    if (!tk.number(nv) || !tk.number(nt) || !tk.number(nc)) return bad("bad size line");
    if (nv < 3 || nt < 1 || nc < 1 || nv > (int64_t(1) << 30) || nt > (int64_t(1) << 30) || nc > (1 << 20))
        return bad("sizes out of range");
    std::vector<double> sigma(nc), xyz(3 * nv);
    std::vector<int32_t> tri(3 * nt), cond(nt);
    for (auto &s : sigma)
        if (!tk.number(s)) return bad("bad conductivity");
    for (auto &x : xyz)
        if (!tk.number(x)) return bad("bad or missing vertex coordinate");
    for (int64_t t = 0; t < nt; ++t) {
        if (!tk.number(tri[3 * t]) || !tk.number(tri[3 * t + 1]) || !tk.number(tri[3 * t + 2]) ||
            !tk.number(cond[t]))
            return bad("bad or missing triangle " + std::to_string(t));
    }
    std::string_view extra;
    if (tk.next(extra)) return bad("trailing data after the last triangle");
    return sie_mesh_load(xyz.data(), nv, tri.data(), nt, cond.data(), sigma.data(), int32_t(nc), out);
}

namespace {

struct UnionFind {
    std::vector<int64_t> p;
    explicit UnionFind(int64_t n) : p(n) { std::iota(p.begin(), p.end(), 0); }
    int64_t find(int64_t a) {
        while (p[a] != a) {
            p[a] = p[p[a]];
            a = p[a];
        }
        return a;
    }
    void unite(int64_t a, int64_t b) {  // the smaller root wins, so a root is its set's minimum
        a = find(a);
        b = find(b);
        if (a == b) return;
        if (a < b) p[b] = a; else p[a] = b;
    }
};

}  // namespace

extern "C" int loop_basis_build(const sie_mesh *m, const sie_port *ports, int32_t np,
                                sie_loops **out, sie_loop_stats *st) {
    if (!m || !out || np < 0 || (np > 0 && !ports))
        return sie::fail(SIE_ERR_ARG, "loop_basis_build: NULL argument");
    *out = nullptr;
    const int64_t nt = m->nt;
    // ---- edges: unique sorted vertex pairs, lexicographic order
    std::vector<std::tuple<int32_t, int32_t, int32_t, int8_t>> half;  // (vmin, vmax, tri, local k)
    half.reserve(3 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            int32_t a = m->tri[3 * t + (k + 1) % 3], b = m->tri[3 * t + (k + 2) % 3];
            if (a > b) std::swap(a, b);
            half.emplace_back(a, b, int32_t(t), int8_t(k));
        }
    std::sort(half.begin(), half.end());
    // ---- contact contraction
    UnionFind uf(nt);
    for (int32_t p = 0; p < np; ++p) {
        const int32_t *sets[2] = {ports[p].src, ports[p].sink};
        int32_t ns[2] = {ports[p].n_src, ports[p].n_sink};
        for (int s = 0; s < 2; ++s) {
            if (ns[s] <= 0 || !sets[s])
                return sie::fail(SIE_ERR_BAD_PORT, "port " + std::to_string(p) + ": empty contact set");
            for (int32_t i = 0; i < ns[s]; ++i) {
                if (sets[s][i] < 0 || sets[s][i] >= nt)
                    return sie::fail(SIE_ERR_BAD_PORT, "port " + std::to_string(p) + ": triangle index out of range");
                uf.unite(sets[s][0], sets[s][i]);
            }
        }
    }
    sie_loops *L = new (std::nothrow) sie_loops;
    if (!L) return sie::fail(SIE_ERR_OOM, "loop_basis_build: out of host memory");
    L->nt = nt;
    L->node_of_tri.resize(nt);
    {
        std::vector<int64_t> rep(nt);
        for (int64_t t = 0; t < nt; ++t) rep[t] = uf.find(t);
        std::vector<int64_t> reps(rep);
        std::sort(reps.begin(), reps.end());
        reps.erase(std::unique(reps.begin(), reps.end()), reps.end());
        for (int64_t t = 0; t < nt; ++t)
            L->node_of_tri[t] = std::lower_bound(reps.begin(), reps.end(), rep[t]) - reps.begin();
        L->n_nodes = int64_t(reps.size());
    }
    // ---- branches in edge order
    for (size_t i = 0; i < half.size();) {
        size_t j = i;
        while (j < half.size() && std::get<0>(half[j]) == std::get<0>(half[i]) &&
               std::get<1>(half[j]) == std::get<1>(half[i]))
            ++j;
        size_t cnt = j - i;
        if (cnt > 2) {
            delete L;
            return sie::fail(SIE_ERR_NONMANIFOLD, "edge (" + std::to_string(std::get<0>(half[i])) + "," +
                                                      std::to_string(std::get<1>(half[i])) + ") shared by " +
                                                      std::to_string(cnt) + " triangles");
        }
        if (cnt == 2) {
            int32_t ta = std::get<2>(half[i]), tb = std::get<2>(half[i + 1]);
            int8_t ka = std::get<3>(half[i]), kb = std::get<3>(half[i + 1]);
            if (ta > tb) { std::swap(ta, tb); std::swap(ka, kb); }
            if (ta == tb) {
                delete L;
                return sie::fail(SIE_ERR_ARG, "triangle " + std::to_string(ta) + " repeats an edge");
            }
            if (L->node_of_tri[ta] != L->node_of_tri[tb]) {
                L->br_tri.push_back(ta);
                L->br_tri.push_back(tb);
                L->br_local.push_back(ka);
                L->br_local.push_back(kb);
            }
        }
        i = j;
    }
    const int64_t nb = int64_t(L->br_tri.size() / 2);
    L->nb = nb;
    L->np = np;
    L->tail.resize(nb + np);
    L->head.resize(nb + np);
    for (int64_t b = 0; b < nb; ++b) {
        L->tail[b] = int32_t(L->node_of_tri[L->br_tri[2 * b]]);
        L->head[b] = int32_t(L->node_of_tri[L->br_tri[2 * b + 1]]);
    }
    for (int32_t p = 0; p < np; ++p) {
        int32_t smin = *std::min_element(ports[p].src, ports[p].src + ports[p].n_src);
        int32_t kmin = *std::min_element(ports[p].sink, ports[p].sink + ports[p].n_sink);
        L->tail[nb + p] = int32_t(L->node_of_tri[kmin]);
        L->head[nb + p] = int32_t(L->node_of_tri[smin]);
        L->port_src.push_back(L->head[nb + p]);
        L->port_sink.push_back(L->tail[nb + p]);
    }
    // ---- adjacency (ascending branch id) and BFS forest
    const int64_t nn = L->n_nodes;
    std::vector<int64_t> deg(nn + 1, 0);
    for (int64_t b = 0; b < nb; ++b) { deg[L->tail[b] + 1]++; deg[L->head[b] + 1]++; }
    for (int64_t i = 0; i < nn; ++i) deg[i + 1] += deg[i];
    std::vector<int32_t> adj_b(2 * nb), fill(deg.begin(), deg.end() - 1);
    std::vector<int32_t> adj_n(2 * nb);
    for (int64_t b = 0; b < nb; ++b) {
        adj_b[fill[L->tail[b]]] = int32_t(b); adj_n[fill[L->tail[b]]++] = L->head[b];
        adj_b[fill[L->head[b]]] = int32_t(b); adj_n[fill[L->head[b]]++] = L->tail[b];
    }
    L->parent.assign(nn, -1);
    L->parent_branch.assign(nn, -1);
    L->comp.assign(nn, -1);
    std::vector<int32_t> depth(nn, 0);
    std::vector<int32_t> bfs_order;
    bfs_order.reserve(nn);
    int32_t ncomp = 0;
    for (int64_t r = 0; r < nn; ++r) {
        if (L->comp[r] >= 0) continue;
        L->comp[r] = ncomp;
        std::deque<int32_t> q{int32_t(r)};
        while (!q.empty()) {
            int32_t u = q.front();
            q.pop_front();
            bfs_order.push_back(u);
            for (int64_t e = deg[u]; e < deg[u + 1]; ++e) {
                int32_t w = adj_n[e];
                if (L->comp[w] < 0) {
                    L->comp[w] = ncomp;
                    L->parent[w] = u;
                    L->parent_branch[w] = adj_b[e];
                    depth[w] = depth[u] + 1;
                    L->depth = std::max<int64_t>(L->depth, depth[w]);
                    q.push_back(w);
                }
            }
        }
        ++ncomp;
    }
    L->n_comp = ncomp;
    for (int32_t p = 0; p < np; ++p) {
        int32_t a = L->tail[nb + p], b = L->head[nb + p];
        if (a == b) {
            delete L;
            return sie::fail(SIE_ERR_BAD_PORT, "port " + std::to_string(p) + ": source and sink are the same node");
        }
        if (L->comp[a] != L->comp[b]) {
            delete L;
            return sie::fail(SIE_ERR_BAD_PORT, "port " + std::to_string(p) + ": source and sink on separate conductors");
        }
    }
    // ---- links and loops
    std::vector<char> twig(nb + np, 0);
    for (int64_t v = 0; v < nn; ++v)
        if (L->parent_branch[v] >= 0) twig[L->parent_branch[v]] = 1;
    L->loop_of_branch.assign(nb + np, -1);
    for (int64_t b = 0; b < nb + np; ++b)
        if (!twig[b]) {
            L->loop_of_branch[b] = int32_t(L->link_branch.size());
            L->link_branch.push_back(int32_t(b));
        }
    L->nl = int64_t(L->link_branch.size());
    L->a_ptr.assign(1, 0);
    std::vector<int32_t> up_w, up_u;
    for (int64_t l = 0; l < L->nl; ++l) {
        int32_t e = L->link_branch[l];
        int32_t u = L->tail[e], w = L->head[e];
        L->a_col.push_back(e);
        L->a_val.push_back(1);
        up_w.clear();
        up_u.clear();
        int32_t x = w, y = u;
        while (depth[x] > depth[y]) { up_w.push_back(x); x = L->parent[x]; }
        while (depth[y] > depth[x]) { up_u.push_back(y); y = L->parent[y]; }
        while (x != y) { up_w.push_back(x); up_u.push_back(y); x = L->parent[x]; y = L->parent[y]; }
        for (int32_t z : up_w) {  // child -> parent
            int32_t t = L->parent_branch[z];
            L->a_col.push_back(t);
            L->a_val.push_back(L->tail[t] == z ? 1 : -1);
        }
        for (int32_t z : up_u) {  // parent -> child
            int32_t t = L->parent_branch[z];
            L->a_col.push_back(t);
            L->a_val.push_back(L->head[t] == z ? 1 : -1);
        }
        L->a_ptr.push_back(int64_t(L->a_col.size()));
    }
    // ---- Euler tour (children in ascending node id) for the device scans
    {
        std::vector<int64_t> cptr(nn + 1, 0);
        for (int64_t v = 0; v < nn; ++v)
            if (L->parent[v] >= 0) cptr[L->parent[v] + 1]++;
        for (int64_t i = 0; i < nn; ++i) cptr[i + 1] += cptr[i];
        std::vector<int32_t> child(cptr[nn]);
        std::vector<int64_t> cf(cptr.begin(), cptr.end() - 1);
        for (int64_t v = 0; v < nn; ++v)
            if (L->parent[v] >= 0) child[cf[L->parent[v]]++] = int32_t(v);
        L->enter.assign(nn, -1);
        L->exit_.assign(nn, -1);
        L->tour_node.assign(2 * nn, 0);
        L->tour_is_enter.assign(2 * nn, 0);
        int32_t pos = 0;
        std::vector<std::pair<int32_t, int64_t>> stack;
        for (int64_t r = 0; r < nn; ++r) {
            if (L->parent[r] >= 0) continue;
            stack.emplace_back(int32_t(r), cptr[r]);
            L->enter[r] = pos;
            L->tour_node[pos] = int32_t(r);
            L->tour_is_enter[pos++] = 1;
            while (!stack.empty()) {
                auto &top = stack.back();
                if (top.second < cptr[top.first + 1]) {
                    int32_t c = child[top.second++];
                    L->enter[c] = pos;
                    L->tour_node[pos] = c;
                    L->tour_is_enter[pos++] = 1;
                    stack.emplace_back(c, cptr[c]);
                } else {
                    L->exit_[top.first] = pos;
                    L->tour_node[pos] = top.first;
                    L->tour_is_enter[pos++] = 0;
                    stack.pop_back();
                }
            }
        }
    }
    // ---- per-node incident links: +1 where the link enters the node (head)
    {
        std::vector<std::vector<std::pair<int32_t, int8_t>>> inc(nn);
        for (int64_t l = 0; l < L->nl; ++l) {
            int32_t e = L->link_branch[l];
            inc[L->head[e]].emplace_back(int32_t(l), int8_t(1));
            inc[L->tail[e]].emplace_back(int32_t(l), int8_t(-1));
        }
        L->nl_ptr.assign(1, 0);
        for (int64_t v = 0; v < nn; ++v) {
            for (auto &pr : inc[v]) { L->nl_loop.push_back(pr.first); L->nl_sign.push_back(pr.second); }
            L->nl_ptr.push_back(int32_t(L->nl_loop.size()));
        }
    }
    if (st) {
        st->n_nodes = nn;
        st->n_branches = nb;
        st->n_comp = ncomp;
        st->n_loops = L->nl;
        st->n_ports = np;
        st->tree_depth = L->depth;
        st->nnz_A = int64_t(L->a_col.size());
    }
    *out = L;
    return SIE_OK;
}

extern "C" void sie_loops_destroy(sie_loops *l) { delete l; }

extern "C" int sie_loops_export(const sie_loops *l, int64_t *row_ptr, int32_t *col, int8_t *val,
                                int32_t *br_tri) {
    if (!l) return sie::fail(SIE_ERR_ARG, "sie_loops_export: NULL loops");
    if (row_ptr) std::memcpy(row_ptr, l->a_ptr.data(), l->a_ptr.size() * sizeof(int64_t));
    if (col) std::memcpy(col, l->a_col.data(), l->a_col.size() * sizeof(int32_t));
    if (val) std::memcpy(val, l->a_val.data(), l->a_val.size() * sizeof(int8_t));
    if (br_tri) std::memcpy(br_tri, l->br_tri.data(), l->br_tri.size() * sizeof(int32_t));
    return SIE_OK;
}
