// Volume, surface and line meshes of the multidimensional solver (Sec. 3.2,
// Table 1): tetrahedra, the cell faces on HABC faces (K^tri triangles), the
// cell edges on domain edges between two HABC faces (K^lin line cells) and the
// corners joining three HABC faces (K^pnt).  Geometric factors of the affine
// maps; Fscale = |grad zeta_f| = sJ/J for the face coordinates zeta_f.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>

#include "setup.h"

namespace dgh {

static const int kTetFace[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
static const int kTriEdge[3][2] = {{0, 1}, {1, 2}, {0, 2}};

static bool inv3(const double A[9], double B[9], double &det) {
    det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (std::fabs(det) < 1e-300) return false;
    const double id = 1.0 / det;
    B[0] = (A[4] * A[8] - A[5] * A[7]) * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = (A[5] * A[6] - A[3] * A[8]) * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = (A[3] * A[7] - A[4] * A[6]) * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return true;
}

bool build_mesh(HostMesh &m, const RefTet &T, const RefTri &F, const RefLine &L, std::string &err) {
    const int64_t K = m.K;
    const int Nfp = T.Nfp;
    (void)F;
    (void)L;
    // bounding box and tolerance
    for (int d = 0; d < 3; ++d) {
        m.lo[d] = 1e300;
        m.hi[d] = -1e300;
    }
    for (int64_t v = 0; v < m.Nv; ++v)
        for (int d = 0; d < 3; ++d) {
            m.lo[d] = std::min(m.lo[d], m.VX[3 * v + d]);
            m.hi[d] = std::max(m.hi[d], m.VX[3 * v + d]);
        }
    double ext = 0;
    for (int d = 0; d < 3; ++d) ext = std::max(ext, m.hi[d] - m.lo[d]);
    const double tol = 1e-9 * std::max(1.0, ext);
    for (int64_t k = 0; k < K; ++k)
        for (int a = 0; a < 4; ++a) {
            const int32_t v = m.EToV[4 * k + a];
            if (v < 0 || v >= m.Nv) {
                err = "cell vertex id out of range";
                return false;
            }
        }
    // ---- 3D geometry
    m.J.resize(K);
    m.drdx.resize(K * 9);
    m.nrm.resize(K * 12);
    m.fscale.resize(K * 4);
    for (int64_t k = 0; k < K; ++k) {
        const double *v0 = &m.VX[3 * m.EToV[4 * k + 0]];
        double Jm[9];
        for (int j = 0; j < 3; ++j) {
            const double *vj = &m.VX[3 * m.EToV[4 * k + 1 + j]];
            for (int d = 0; d < 3; ++d) Jm[3 * d + j] = 0.5 * (vj[d] - v0[d]);  // dx_d / dr_j
        }
        double G[9], det;
        if (!inv3(Jm, G, det) || std::fabs(det) < 1e-14 * ext * ext * ext) {
            err = "degenerate tetrahedron " + std::to_string(k);
            return false;
        }
        m.J[k] = det;
        for (int q = 0; q < 9; ++q) m.drdx[9 * k + q] = G[q];  // G[j][i] = dr_j/dx_i
        const double *g = &m.drdx[9 * k];
        double z[4][3];
        for (int i = 0; i < 3; ++i) {
            z[0][i] = -g[6 + i];                 // -grad t
            z[1][i] = -g[3 + i];                 // -grad s
            z[2][i] = g[i] + g[3 + i] + g[6 + i];  // +grad (r+s+t)
            z[3][i] = -g[i];                     // -grad r
        }
        for (int f = 0; f < 4; ++f) {
            const double nn = std::sqrt(z[f][0] * z[f][0] + z[f][1] * z[f][1] + z[f][2] * z[f][2]);
            m.fscale[4 * k + f] = nn;
            for (int i = 0; i < 3; ++i) m.nrm[12 * k + 3 * f + i] = z[f][i] / nn;
        }
    }
    // ---- face connectivity by sorted vertex triples
    std::vector<std::tuple<int32_t, int32_t, int32_t, int64_t>> faces(K * 4);
    for (int64_t k = 0; k < K; ++k)
        for (int f = 0; f < 4; ++f) {
            int32_t v[3] = {m.EToV[4 * k + kTetFace[f][0]], m.EToV[4 * k + kTetFace[f][1]], m.EToV[4 * k + kTetFace[f][2]]};
            std::sort(v, v + 3);
            faces[4 * k + f] = std::make_tuple(v[0], v[1], v[2], 4 * k + f);
        }
    std::sort(faces.begin(), faces.end());
    m.nbr.assign(K * 4, -1);
    m.nbrSigma.assign(K * 4, 0);
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && std::get<0>(faces[j]) == std::get<0>(faces[i]) &&
               std::get<1>(faces[j]) == std::get<1>(faces[i]) && std::get<2>(faces[j]) == std::get<2>(faces[i]))
            ++j;
        if (j - i > 2) {
            err = "non-manifold mesh: a face is shared by more than two cells";
            return false;
        }
        if (j - i == 2) {
            const int64_t a = std::get<3>(faces[i]), b = std::get<3>(faces[i + 1]);
            m.nbr[a] = b;
            m.nbr[b] = a;
        }
        i = j;
    }
    // vertex permutation codes: own face vertex q is vertex kSigma[code][q] of the neighbour face
    for (int64_t gf = 0; gf < K * 4; ++gf) {
        const int64_t nb = m.nbr[gf];
        if (nb < 0) continue;
        const int64_t k = gf / 4, k2 = nb / 4;
        const int f = int(gf % 4), f2 = int(nb % 4);
        int pos[3];
        for (int q = 0; q < 3; ++q) {
            pos[q] = -1;
            for (int q2 = 0; q2 < 3; ++q2)
                if (m.EToV[4 * k + kTetFace[f][q]] == m.EToV[4 * k2 + kTetFace[f2][q2]]) pos[q] = q2;
        }
        int code = -1;
        for (int sg = 0; sg < 6; ++sg)
            if (kSigma[sg][0] == pos[0] && kSigma[sg][1] == pos[1] && kSigma[sg][2] == pos[2]) code = sg;
        if (code < 0) {
            err = "face matching failed";
            return false;
        }
        m.nbrSigma[gf] = int8_t(code);
    }
    // ---- boundary faces and their domain face
    m.bfaceOf.assign(K * 4, -1);
    for (int64_t gf = 0; gf < K * 4; ++gf) {
        if (m.nbr[gf] >= 0) continue;
        const int64_t k = gf / 4;
        const int f = int(gf % 4);
        int dom = -1;
        for (int a = 0; a < 3; ++a) {
            bool lo = true, hi = true;
            for (int q = 0; q < 3; ++q) {
                const double x = m.VX[3 * m.EToV[4 * k + kTetFace[f][q]] + a];
                lo = lo && std::fabs(x - m.lo[a]) < tol;
                hi = hi && std::fabs(x - m.hi[a]) < tol;
            }
            if (lo) dom = 2 * a;
            if (hi) dom = 2 * a + 1;
        }
        if (dom < 0) {
            err = "a boundary face is not on the cuboid boundary";
            return false;
        }
        m.bfaceOf[gf] = int64_t(m.bface.size());
        m.bface.push_back(gf);
        m.bfaceDom.push_back(dom);
    }
    // ---- triangles: HABC boundary faces in increasing (cell, face)
    for (size_t b = 0; b < m.bface.size(); ++b)
        if (m.face_habc(m.bfaceDom[b])) m.triBface.push_back(int64_t(b));
    const int64_t Tn = m.Ktri = int64_t(m.triBface.size());
    m.triDom.resize(Tn);
    m.triV.resize(Tn * 3);
    m.triAxes.resize(Tn * 2);
    m.drdx2.resize(Tn * 4);
    m.nrm2.resize(Tn * 6);
    m.fscale2.resize(Tn * 3);
    for (int64_t t = 0; t < Tn; ++t) {
        const int64_t gf = m.bface[m.triBface[t]];
        const int64_t k = gf / 4;
        const int f = int(gf % 4);
        const int d = m.bfaceDom[m.triBface[t]];
        m.triDom[t] = d;
        const int ax0 = (d / 2 == 0) ? 1 : 0, ax1 = (d / 2 == 2) ? 1 : 2;
        m.triAxes[2 * t] = ax0;
        m.triAxes[2 * t + 1] = ax1;
        double w[3][2];
        for (int q = 0; q < 3; ++q) {
            const int32_t v = m.EToV[4 * k + kTetFace[f][q]];
            m.triV[3 * t + q] = v;
            w[q][0] = m.VX[3 * v + ax0];
            w[q][1] = m.VX[3 * v + ax1];
        }
        const double a = 0.5 * (w[1][0] - w[0][0]), b = 0.5 * (w[2][0] - w[0][0]);  // dx/dr, dx/ds
        const double c = 0.5 * (w[1][1] - w[0][1]), dd = 0.5 * (w[2][1] - w[0][1]);  // dy/dr, dy/ds
        const double det = a * dd - b * c;
        // [dr/dx dr/dy; ds/dx ds/dy]
        const double rx = dd / det, ry = -b / det, sx = -c / det, sy = a / det;
        double *g = &m.drdx2[4 * t];
        g[0] = rx;
        g[1] = ry;
        g[2] = sx;
        g[3] = sy;
        const double z[3][2] = {{-sx, -sy}, {rx + sx, ry + sy}, {-rx, -ry}};
        for (int e = 0; e < 3; ++e) {
            const double nn = std::sqrt(z[e][0] * z[e][0] + z[e][1] * z[e][1]);
            m.fscale2[3 * t + e] = nn;
            m.nrm2[6 * t + 2 * e] = z[e][0] / nn;
            m.nrm2[6 * t + 2 * e + 1] = z[e][1] / nn;
        }
    }
    // triangle edges: key (sorted vertex pair, domain face)
    std::map<std::tuple<int32_t, int32_t, int>, std::vector<int64_t>> ekeys;
    for (int64_t t = 0; t < Tn; ++t)
        for (int e = 0; e < 3; ++e) {
            int32_t a = m.triV[3 * t + kTriEdge[e][0]], b = m.triV[3 * t + kTriEdge[e][1]];
            if (a > b) std::swap(a, b);
            ekeys[std::make_tuple(a, b, m.triDom[t])].push_back(3 * t + e);
        }
    m.nbr2.assign(Tn * 3, -1);
    m.flip2.assign(Tn * 3, 0);
    m.edgeDom.assign(Tn * 3, -1);
    for (auto &kv : ekeys) {
        auto &v = kv.second;
        if (v.size() > 2) {
            err = "surface mesh is non-manifold";
            return false;
        }
        if (v.size() == 2) {
            const int64_t e1 = v[0], e2 = v[1];
            m.nbr2[e1] = e2;
            m.nbr2[e2] = e1;
            const int32_t a1 = m.triV[3 * (e1 / 3) + kTriEdge[e1 % 3][0]];
            const int32_t a2 = m.triV[3 * (e2 / 3) + kTriEdge[e2 % 3][0]];
            m.flip2[e1] = m.flip2[e2] = (a1 != a2);
        } else {
            const int64_t ge = v[0], t = ge / 3;
            const int e = int(ge % 3);
            const int32_t va = m.triV[3 * t + kTriEdge[e][0]], vb = m.triV[3 * t + kTriEdge[e][1]];
            int found = -1;
            for (int b = 0; b < 3; ++b) {
                if (b == m.triDom[t] / 2) continue;
                const double xa = m.VX[3 * va + b], xb = m.VX[3 * vb + b];
                if (std::fabs(xa - m.lo[b]) < tol && std::fabs(xb - m.lo[b]) < tol) found = 2 * b;
                if (std::fabs(xa - m.hi[b]) < tol && std::fabs(xb - m.hi[b]) < tol) found = 2 * b + 1;
            }
            if (found < 0) {
                err = "open triangle edge inside a domain face";
                return false;
            }
            m.edgeDom[ge] = found;
        }
    }
    // ---- line cells: by face-A triangle, then local edge
    for (int s = 0; s < 2; ++s) {
        m.linTri[s].clear();
        m.linEdge[s].clear();
        m.linRev[s].clear();
    }
    for (int64_t t = 0; t < Tn; ++t)
        for (int e = 0; e < 3; ++e) {
            const int B = m.edgeDom[3 * t + e];
            const int A = m.triDom[t];
            if (B < 0 || B < A || !m.face_habc(B)) continue;
            int32_t va = m.triV[3 * t + kTriEdge[e][0]], vb = m.triV[3 * t + kTriEdge[e][1]];
            const int g = 3 - A / 2 - B / 2;
            const bool rev = m.VX[3 * va + g] > m.VX[3 * vb + g];
            int32_t lo = rev ? vb : va, hi = rev ? va : vb;
            auto it = ekeys.find(std::make_tuple(std::min(va, vb), std::max(va, vb), B));
            if (it == ekeys.end() || it->second.size() != 1) {
                err = "edge partner on face B not found";
                return false;
            }
            const int64_t geB = it->second[0], tB = geB / 3;
            const int eB = int(geB % 3);
            const int32_t vaB = m.triV[3 * tB + kTriEdge[eB][0]];
            m.linTri[0].push_back(t);
            m.linEdge[0].push_back(e);
            m.linRev[0].push_back(rev);
            m.linTri[1].push_back(tB);
            m.linEdge[1].push_back(eB);
            m.linRev[1].push_back(vaB != lo);
            m.linA.push_back(A);
            m.linB.push_back(B);
            m.linAxis.push_back(g);
            m.linV.push_back(lo);
            m.linV.push_back(hi);
            m.J1.push_back(0.5 * (m.VX[3 * hi + g] - m.VX[3 * lo + g]));
        }
    const int64_t Ln = m.Klin = int64_t(m.linA.size());
    m.nbr1.assign(Ln * 2, -1);
    m.endDom.assign(Ln * 2, -1);
    std::map<std::tuple<int, int, int32_t>, std::vector<int64_t>> vend;
    for (int64_t l = 0; l < Ln; ++l)
        for (int end = 0; end < 2; ++end) vend[std::make_tuple(m.linA[l], m.linB[l], m.linV[2 * l + end])].push_back(2 * l + end);
    std::map<std::tuple<int, int, int>, std::vector<int64_t>> cornerEnds;
    for (auto &kv : vend) {
        auto &v = kv.second;
        if (v.size() == 2) {
            m.nbr1[v[0]] = v[1];
            m.nbr1[v[1]] = v[0];
        } else if (v.size() == 1) {
            const int64_t l = v[0] / 2;
            const int g = m.linAxis[l];
            const double x = m.VX[3 * m.linV[v[0]] + g];
            int X = -1;
            if (std::fabs(x - m.lo[g]) < tol) X = 2 * g;
            if (std::fabs(x - m.hi[g]) < tol) X = 2 * g + 1;
            if (X < 0) {
                err = "line chain ends inside a domain edge";
                return false;
            }
            m.endDom[v[0]] = X;
            int fs[3] = {m.linA[l], m.linB[l], X};
            std::sort(fs, fs + 3);
            cornerEnds[std::make_tuple(fs[0], fs[1], fs[2])].push_back(v[0]);
        } else {
            err = "line mesh is not a chain";
            return false;
        }
    }
    m.corners.clear();
    for (auto &kv : cornerEnds) {
        const int X = std::get<0>(kv.first), Y = std::get<1>(kv.first), Z = std::get<2>(kv.first);
        if (!(m.face_habc(X) && m.face_habc(Y) && m.face_habc(Z))) continue;
        if (kv.second.size() != 3) {
            err = "a corner must join three line cells";
            return false;
        }
        HostMesh::Corner c;
        c.faces[0] = X;
        c.faces[1] = Y;
        c.faces[2] = Z;
        for (int64_t le : kv.second) {
            const int64_t l = le / 2;
            int slot = -1;
            if (m.linA[l] == Y && m.linB[l] == Z) slot = 0;
            if (m.linA[l] == X && m.linB[l] == Z) slot = 1;
            if (m.linA[l] == X && m.linB[l] == Y) slot = 2;
            if (slot < 0) {
                err = "corner edge bookkeeping failed";
                return false;
            }
            c.line[slot] = l;
            c.end[slot] = int(le % 2);
        }
        m.corners.push_back(c);
    }
    // p = 0 flags per entity
    m.bfaceDir.assign(m.bface.size(), 0);
    for (size_t b = 0; b < m.bface.size(); ++b) m.bfaceDir[b] = m.bc[m.bfaceDom[b]] == BC_DIRICHLET;
    m.edgeDir.assign(size_t(Tn) * 3, 0);
    for (int64_t ge = 0; ge < Tn * 3; ++ge)
        if (m.edgeDom[ge] >= 0) m.edgeDir[ge] = m.bc[m.edgeDom[ge]] == BC_DIRICHLET;
    m.endDir.assign(size_t(Ln) * 2, 0);
    for (int64_t le = 0; le < Ln * 2; ++le)
        if (m.endDom[le] >= 0) m.endDir[le] = m.bc[m.endDom[le]] == BC_DIRICHLET;
    (void)Nfp;
    return true;
}

void merge_meshes(const std::vector<HostMesh> &parts, HostMesh &o) {
    o = HostMesh();
    o.N = parts.empty() ? 0 : parts[0].N;
    o.P = parts.empty() ? 0 : parts[0].P;
    for (int d = 0; d < 6; ++d) o.bc[d] = BC_HABC;
    for (int d = 0; d < 3; ++d) {
        o.lo[d] = 1e300;
        o.hi[d] = -1e300;
    }
    int64_t vOff = 0, kOff = 0, bOff = 0, tOff = 0, lOff = 0;
    auto app = [](auto &dst, const auto &src) { dst.insert(dst.end(), src.begin(), src.end()); };
    for (const HostMesh &m : parts) {
        for (int d = 0; d < 3; ++d) {
            o.lo[d] = std::min(o.lo[d], m.lo[d]);
            o.hi[d] = std::max(o.hi[d], m.hi[d]);
        }
        app(o.VX, m.VX);
        for (int32_t v : m.EToV) o.EToV.push_back(int32_t(v + vOff));
        app(o.c, m.c);
        app(o.rho, m.rho);
        app(o.J, m.J);
        app(o.drdx, m.drdx);
        app(o.nrm, m.nrm);
        app(o.fscale, m.fscale);
        for (int64_t x : m.nbr) o.nbr.push_back(x >= 0 ? x + 4 * kOff : -1);
        app(o.nbrSigma, m.nbrSigma);
        for (int64_t x : m.bface) o.bface.push_back(x + 4 * kOff);
        app(o.bfaceDom, m.bfaceDom);
        for (int64_t x : m.bfaceOf) o.bfaceOf.push_back(x >= 0 ? x + bOff : -1);
        app(o.bfaceDir, m.bfaceDir);
        for (int64_t x : m.triBface) o.triBface.push_back(x + bOff);
        app(o.triDom, m.triDom);
        for (int32_t v : m.triV) o.triV.push_back(int32_t(v + vOff));
        app(o.triAxes, m.triAxes);
        app(o.drdx2, m.drdx2);
        app(o.nrm2, m.nrm2);
        app(o.fscale2, m.fscale2);
        for (int64_t x : m.nbr2) o.nbr2.push_back(x >= 0 ? x + 3 * tOff : -1);
        app(o.flip2, m.flip2);
        app(o.edgeDom, m.edgeDom);
        app(o.edgeDir, m.edgeDir);
        for (int s = 0; s < 2; ++s) {
            for (int64_t x : m.linTri[s]) o.linTri[s].push_back(x + tOff);
            app(o.linEdge[s], m.linEdge[s]);
            app(o.linRev[s], m.linRev[s]);
        }
        app(o.linA, m.linA);
        app(o.linB, m.linB);
        app(o.linAxis, m.linAxis);
        for (int32_t v : m.linV) o.linV.push_back(int32_t(v + vOff));
        app(o.J1, m.J1);
        for (int64_t x : m.nbr1) o.nbr1.push_back(x >= 0 ? x + 2 * lOff : -1);
        app(o.endDom, m.endDom);
        app(o.endDir, m.endDir);
        for (HostMesh::Corner c : m.corners) {
            for (int q = 0; q < 3; ++q) c.line[q] += lOff;
            o.corners.push_back(c);
        }
        if (m.dtCell.empty()) {
            o.dtCell.insert(o.dtCell.end(), size_t(m.K), 0.0);
        } else {
            app(o.dtCell, m.dtCell);
        }
        vOff += m.Nv;
        kOff += m.K;
        bOff += int64_t(m.bface.size());
        tOff += m.Ktri;
        lOff += m.Klin;
    }
    o.Nv = vOff;
    o.K = kOff;
    o.Ktri = tOff;
    o.Klin = lOff;
}

double dt_rule(const HostMesh &m, double cfl) {
    double best = 1e300;
    for (int64_t k = 0; k < m.K; ++k) {
        double fmax = 0;
        for (int f = 0; f < 4; ++f) fmax = std::max(fmax, m.fscale[4 * k + f]);
        best = std::min(best, 1.0 / (m.c[k] * (m.N + 1) * (m.N + 1) * fmax));
    }
    return cfl * best;
}

// ------------------------------------------------------------------ HABC operators
// Edge (Sec. 3.1, eqs. proc:edgeBC1-2): with Q = r^- + r^+,
//   r^-_A,a = (1/M) sum_b c_b (p*_ab + (C_ba - 1) Q_A,a + C_ab Q_B,b)
//   r^-_B,b = (1/M) sum_a c_a (p*_ab + C_ba Q_A,a + (C_ab - 1) Q_B,b)
// i.e. x = G (x + rp) + F ps  =>  x = (I-G)^{-1} G rp + (I-G)^{-1} F ps.
// Corner (eqs. proc:cornerBC1-3) similarly x = G (x + rp)  =>  x = (I-G)^{-1} G rp.
bool build_habc(int P, HabcOps &o, std::string &err) {
    o.P = P;
    o.M = 2 * P + 1;
    o.c.resize(P);
    for (int n = 1; n <= P; ++n) {
        const double tn = std::tan(n * M_PI / o.M);
        o.c[n - 1] = tn * tn;
    }
    if (P == 0) return true;
    const double iM = 1.0 / o.M;
    const auto &c = o.c;
    auto C2 = [&](int a, int b) { return (1.0 + c[a]) / (1.0 + c[a] + c[b]); };
    Mat G(2 * P, 2 * P), Fm(2 * P, P * P);
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            const int s = a + P * b;
            // row of face A set a
            G(a, a) += iM * c[b] * (C2(b, a) - 1.0);
            G(a, P + b) += iM * c[b] * C2(a, b);
            Fm(a, s) += iM * c[b];
            // row of face B set b
            G(P + b, a) += iM * c[a] * C2(b, a);
            G(P + b, P + b) += iM * c[a] * (C2(a, b) - 1.0);
            Fm(P + b, s) += iM * c[a];
        }
    Mat IG(2 * P, 2 * P), IGi;
    for (int i = 0; i < 2 * P; ++i)
        for (int j = 0; j < 2 * P; ++j) IG(i, j) = (i == j ? 1.0 : 0.0) - G(i, j);
    if (!invert(IG, IGi)) {
        err = "edge system is singular";
        return false;
    }
    o.H1 = matmul(IGi, G);
    o.H2 = matmul(IGi, Fm);
    {
        Mat chk = matmul(IG, IGi);
        double r = 0;
        for (int i = 0; i < 2 * P; ++i)
            for (int j = 0; j < 2 * P; ++j) r = std::max(r, std::fabs(chk(i, j) - (i == j)));
        o.residual_edge = r;
    }
    // corner: blocks YZ (index j + P k), XZ (i + P k), XY (i + P j)
    const int n = P * P;
    Mat Gc(3 * n, 3 * n);
    auto C3 = [&](int i, int j, int k) { return (1.0 + c[i]) / (1.0 + c[i] + c[j] + c[k]); };
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j)
            for (int k = 0; k < P; ++k) {
                const int yz = j + P * k, xz = n + i + P * k, xy = 2 * n + i + P * j;
                // p_ijk - p_0jk etc. with p_ijk = C_ijk p_0jk + C_jki p_i0k + C_kij p_ij0
                const double cijk = C3(i, j, k), cjki = C3(j, k, i), ckij = C3(k, i, j);
                Gc(yz, yz) += iM * c[i] * (cijk - 1.0);
                Gc(yz, xz) += iM * c[i] * cjki;
                Gc(yz, xy) += iM * c[i] * ckij;
                Gc(xz, yz) += iM * c[j] * cijk;
                Gc(xz, xz) += iM * c[j] * (cjki - 1.0);
                Gc(xz, xy) += iM * c[j] * ckij;
                Gc(xy, yz) += iM * c[k] * cijk;
                Gc(xy, xz) += iM * c[k] * cjki;
                Gc(xy, xy) += iM * c[k] * (ckij - 1.0);
            }
    Mat IGc(3 * n, 3 * n), IGci;
    for (int i = 0; i < 3 * n; ++i)
        for (int j = 0; j < 3 * n; ++j) IGc(i, j) = (i == j ? 1.0 : 0.0) - Gc(i, j);
    if (!invert(IGc, IGci)) {
        err = "corner system is singular";
        return false;
    }
    o.Hc = matmul(IGci, Gc);
    {
        Mat chk = matmul(IGc, IGci);
        double r = 0;
        for (int i = 0; i < 3 * n; ++i)
            for (int j = 0; j < 3 * n; ++j) r = std::max(r, std::fabs(chk(i, j) - (i == j)));
        o.residual_corner = r;
    }
    return true;
}

}  // namespace dgh
