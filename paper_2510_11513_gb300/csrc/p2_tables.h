// Exact element tables of the second-order (ten-node) tetrahedron, shared by
// the device solve and host set-up (and compiled on its own by a host test).
// Nodes: vertices 0..3, then the midpoints of the edges (0,1) (0,2) (0,3) (1,2)
// (1,3) (2,3).  Values are exact rationals from int lambda^a dV = 6 V a! / (|a| + 3)!
// and int lambda^a dA = 2 A a! / (|a| + 2)!.
#pragma once

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

// Face nodes of face f: its three vertices ascending, then its three edges in
// edge order; in that order the face mass table is the same for every face.
__host__ __device__ constexpr int p2_face_node(int f, int b)
{
    constexpr int FN[4][6] = {{1, 2, 3, 7, 8, 9}, {0, 2, 3, 5, 6, 9}, {0, 1, 3, 4, 6, 8}, {0, 1, 2, 4, 5, 7}};
    return FN[f][b];
}

__host__ __device__ constexpr int p2_edge_end(int e, int k)
{
    constexpr int E[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    return E[e][k];
}

// p_i = int phi_i / V
__host__ __device__ constexpr double p2_p(int i) { return i < 4 ? -1.0 / 20.0 : 1.0 / 5.0; }

// P_im = int phi_i lambda_m / V
__host__ __device__ constexpr double p2_P(int i, int m)
{
    return i < 4 ? (i == m ? 0.0 : -1.0 / 60.0)
                 : ((p2_edge_end(i - 4, 0) == m || p2_edge_end(i - 4, 1) == m) ? 1.0 / 15.0 : 1.0 / 30.0);
}

// Mh_ij = int phi_i phi_j / V
__host__ __device__ constexpr double p2_M(int i, int j)
{
    if (i < 4 && j < 4) return i == j ? 1.0 / 70.0 : 1.0 / 420.0;
    if (i >= 4 && j >= 4) {
        if (i == j) return 8.0 / 105.0;
        const int a = p2_edge_end(i - 4, 0), b = p2_edge_end(i - 4, 1);
        const int c = p2_edge_end(j - 4, 0), d = p2_edge_end(j - 4, 1);
        return (a == c || a == d || b == c || b == d) ? 4.0 / 105.0 : 2.0 / 105.0;
    }
    const int v = i < 4 ? i : j, e = i < 4 ? j - 4 : i - 4;
    return (p2_edge_end(e, 0) == v || p2_edge_end(e, 1) == v) ? -1.0 / 105.0 : -1.0 / 70.0;
}

// Fh_bc = int_f phi_b phi_c / A_f in face node order (vertices 0..2, edges 3..5;
// face edge 3 joins face vertices 0,1, edge 4 joins 0,2, edge 5 joins 1,2)
__host__ __device__ constexpr double p2_F(int b, int c)
{
    if (b < 3 && c < 3) return b == c ? 1.0 / 30.0 : -1.0 / 180.0;
    if (b >= 3 && c >= 3) return b == c ? 8.0 / 45.0 : 4.0 / 45.0;
    const int v = b < 3 ? b : c, e = b < 3 ? c : b;
    // the face edge opposite face vertex v: vertex 0 <-> edge 5, 1 <-> 4, 2 <-> 3
    return e == 5 - v ? -1.0 / 45.0 : 0.0;
}

