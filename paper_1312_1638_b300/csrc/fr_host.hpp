// Host-side set-up of the FR discretisation: standard elements, operator
// matrices (App. A), element mappings / metric terms (Sec. 2) and flux-point
// pairing (Sec. 2, lookup table).  Plain C++17, no CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace fr {

enum { ET_QUAD = 0, ET_TRI = 1, ET_HEX = 2 };

// A standard element of one type at order p (Sec. 2).
struct ElemType {
    int etype = 0, p = 0, ndims = 0, nupts = 0, nfpts = 0, nfaces = 0, nfp_face = 0;
    std::vector<double> upts;    // [nupts][ndims]
    std::vector<double> fpts;    // [nfpts][ndims]
    std::vector<double> fnorm;   // [nfpts][ndims] unit outward reference normals
    std::vector<int> fface;      // [nfpts] face of each flux point
    std::vector<double> gl;      // 1D Gauss-Legendre nodes (p+1)
    std::vector<double> glw;     // and weights
    // Operator matrices, row-major FP64 (App. A).
    std::vector<double> M0;      // nfpts x nupts
    std::vector<double> M1;      // nupts x ndims*nupts
    std::vector<double> M2;      // nfpts x ndims*nupts
    std::vector<double> M3;      // nupts x nfpts
    std::vector<double> M4;      // ndims*nupts x nupts
    std::vector<double> M6;      // ndims*nupts x nfpts
    std::vector<double> M46;     // M4 - M6 M0   (ndims*nupts x nupts)
    std::vector<double> M132;    // M1 - M3 M2   (nupts x ndims*nupts)
    std::vector<double> qw;      // quadrature weight of each solution point (reference element)
    // coefficients of the nodal basis in monomials (triangles only), [nb][nupts]
    std::vector<long double> tri_coef;

    // nodal basis values l_rho(x) [nupts] and gradients [ndims][nupts] at one point
    void nodal(const long double* x, long double* val, long double* grad) const;
};

// correction: 0 = DG, 1 = SD, 2 = HU (VCJH eta = 0, p/(p+1), (p+1)/p; tensor elements)
bool build_element(int etype, int p, ElemType& el, std::string& err, int correction = 0);

// Reference coordinates of the centre of face f and the map from face
// parameters (t) or (a, b) to reference coordinates.
void face_point(int etype, int f, const long double* par, long double* x);

// Element mapping: shape functions (values [nn], derivatives [ndims][nn]).
bool shape_functions(int etype, int nnodes, const long double* x, long double* N,
                     long double* dN);

struct HostBlock {
    int etype = 0, nnodes = 0;
    int64_t nelem = 0;
    const ElemType* el = nullptr;
    std::vector<double> nodes;   // [nelem][nnodes][ndims]
    // shape-function tables of the element mapping (same for every element)
    std::vector<double> Nu, dNu; // at solution points: [nupts][nnodes], [nupts][ndims][nnodes]
    std::vector<double> Nf, dNf; // at flux points
    std::vector<double> Nc;      // at face centres: [nfaces][nnodes]
};

// Fill the shape-function tables of a block (after el, etype, nnodes are set).
bool prepare_block(HostBlock& blk);

struct HostPair {                // one interior flux-point pair
    int32_t bL, fL, bR, fR;
    int64_t nL, nR;
    double nrm[3];               // unit physical normal of the L side
    double magL, magR;           // J^(f) n^(f) on each side
};

struct HostBnd {                 // one boundary flux point
    int32_t b, f, bctype;
    int64_t n;
    double nrm[3];
    double mag;
};

// Metric terms at solution points of one element: adj(J) [npts][ndims][ndims]
// (row-major i,j) and det J [npts].
bool element_metrics(const HostBlock& blk, int64_t e, double* adj, double* det);

// Pair every flux point of the mesh.  Fails on unmatched / doubly matched
// points and on boundary faces that are also paired.
bool pair_mesh(int ndims, const std::vector<HostBlock>& blocks, const int64_t* bfaces,
               int64_t nbfaces, const double* periodic, int nperiodic,
               std::vector<HostPair>& pairs, std::vector<HostBnd>& bnds, std::string& err);

}  // namespace fr
