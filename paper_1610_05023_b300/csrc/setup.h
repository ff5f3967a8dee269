// Host-side set-up of the solver (FP64): reference elements, meshes, maps,
// geometric factors and the HABC solution operators.  Everything here runs
// once in dgh_create(); the result is packed into device arrays by api.cu.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace dgh {

// Dense row-major matrix (FP64).
struct Mat {
    int rows = 0, cols = 0;
    std::vector<double> a;
    Mat() = default;
    Mat(int r, int c) : rows(r), cols(c), a(size_t(r) * c, 0.0) {}
    double &operator()(int i, int j) { return a[size_t(i) * cols + j]; }
    double operator()(int i, int j) const { return a[size_t(i) * cols + j]; }
};
Mat matmul(const Mat &A, const Mat &B);
Mat transpose(const Mat &A);
bool invert(const Mat &A, Mat &Ainv);  // Gauss-Jordan, partial pivoting

// ---------------------------------------------------------------- elements
struct RefLine {
    int N = 0, Np = 0;
    std::vector<double> r;
    Mat V, Dr, LIFT, M;  // LIFT: Np x 2 (ends r=-1, r=+1)
};
struct RefTri {
    int N = 0, Np = 0, Nfp = 0;
    std::vector<double> r, s;
    Mat V, Dr, Ds, LIFT, M;                 // LIFT: Np x 3*Nfp
    std::vector<std::vector<int>> Fmask;    // 3 x Nfp, edge nodes run from the edge's first to second vertex
};
struct RefTet {
    int N = 0, Np = 0, Nfp = 0;
    std::vector<double> r, s, t;
    Mat V, Dr, Ds, Dt, LIFT, M;             // LIFT: Np x 4*Nfp
    std::vector<std::vector<int>> Fmask;    // 4 x Nfp
    // node permutation of a face under a permutation of its three vertices:
    // facePerm[sigma][m] = index of the node that sits where node m sits
    // once vertex i of this face is identified with vertex sigmaTab[sigma][i]
    // of the neighbouring face.
    std::vector<std::vector<int>> facePerm; // 6 x Nfp
};
extern const int kSigma[6][3];

std::vector<double> gll_points(int N);
double warp_alpha_tet(int N);
void build_line(int N, RefLine &out);
void build_tri(int N, double alpha, RefTri &out);
bool build_tet(int N, RefTet &out, std::string &err);
// l_n(r,s,t) of the nodal basis at one point
std::vector<double> tet_interp_row(const RefTet &T, double r, double s, double t);

// ---------------------------------------------------------------- mesh
enum { BC_HABC = 0, BC_DIRICHLET = 1 };

struct HostMesh {
    int N = 0, P = 0;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    int64_t K = 0, Nv = 0;
    std::vector<double> VX;        // Nv*3
    std::vector<int32_t> EToV;     // K*4
    std::vector<double> c, rho;    // K
    double lo[3], hi[3];
    // 3D geometry
    std::vector<double> J;         // K (signed)
    std::vector<double> drdx;      // K*9, [k][j][i] = d r_j / d x_i
    std::vector<double> nrm;       // K*4*3 outward unit normals
    std::vector<double> fscale;    // K*4
    std::vector<int64_t> nbr;      // K*4 neighbour global face id (k'*4+f') or -1
    std::vector<int8_t> nbrSigma;  // K*4 vertex permutation code (0..5)
    // boundary faces (ascending global face id)
    std::vector<int64_t> bface;    // global face id
    std::vector<int> bfaceDom;     // domain face 0..5
    std::vector<int64_t> bfaceOf;  // K*4 -> boundary index or -1
    // 2D
    int64_t Ktri = 0;
    std::vector<int64_t> triBface; // boundary index of each triangle
    std::vector<int> triDom;
    std::vector<int32_t> triV;     // Ktri*3 vertex ids (cell face order)
    std::vector<int> triAxes;      // Ktri*2 in-plane axes
    std::vector<double> drdx2;     // Ktri*4  [t][j][i]
    std::vector<double> nrm2;      // Ktri*3*2
    std::vector<double> fscale2;   // Ktri*3
    std::vector<int64_t> nbr2;     // Ktri*3 neighbour (t'*3+e') or -1
    std::vector<int8_t> flip2;     // Ktri*3 neighbour edge runs the other way
    std::vector<int> edgeDom;      // Ktri*3 adjacent domain face for open edges, -1 else
    // 1D
    int64_t Klin = 0;
    std::vector<int64_t> linTri[2]; // face A / face B triangle
    std::vector<int> linEdge[2];    // local edge of that triangle
    std::vector<int8_t> linRev[2];  // triangle edge runs against +axis
    std::vector<int> linA, linB, linAxis;
    std::vector<int32_t> linV;      // Klin*2, vertex ids ordered along +axis
    std::vector<double> J1;         // Klin
    std::vector<int64_t> nbr1;      // Klin*2 neighbour (l'*2+end') or -1
    std::vector<int> endDom;        // Klin*2 third face at a domain corner, -1 else
    // 0D
    struct Corner { int faces[3]; int64_t line[3]; int end[3]; };  // line[0]: YZ edge, [1]: XZ, [2]: XY
    std::vector<Corner> corners;
    // p = 0 flags resolved per entity (a batch of problems has one bc[] per problem)
    std::vector<int8_t> bfaceDir;  // per boundary face
    std::vector<int8_t> edgeDir;   // per triangle edge (open edges only)
    std::vector<int8_t> endDir;    // per line end (corner ends only)
    std::vector<double> dtCell;    // per-cell time step (batches); empty: one time step for all
    bool face_habc(int d) const { return bc[d] == BC_HABC && P >= 1; }
};

// Disjoint union of meshes of the same N and P (a batch of independent
// problems): indices are offset, per-entity flags and time steps kept.
void merge_meshes(const std::vector<HostMesh> &parts, HostMesh &out);

// Builds all meshes; returns false with a message on invalid input.
bool build_mesh(HostMesh &m, const RefTet &T, const RefTri &F, const RefLine &L, std::string &err);
double dt_rule(const HostMesh &m, double cfl);

// ---------------------------------------------------------------- HABC
struct HabcOps {
    int P = 0, M = 1;
    std::vector<double> c;     // P
    // edge: x = H1 [rpA; rpB] + H2 ps   (x = [rmA; rmB], ps indexed s = a + P b)
    Mat H1, H2;                // 2P x 2P, 2P x P^2
    // corner: x = Hc rp, x / rp = [YZ (s=j+P k); XZ (s=i+P k); XY (s=i+P j)]
    Mat Hc;                    // 3P^2 x 3P^2
    double residual_edge = 0.0, residual_corner = 0.0;  // |A Ainv - I|
};
bool build_habc(int P, HabcOps &ops, std::string &err);

}  // namespace dgh
