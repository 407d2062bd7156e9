// Force-constant files (host only, no GPU): the third- and fourth-order inputs of the paper's program
// (Appendix A: FORCE_CONSTANTS_4TH beside ShengBTE's FORCE_CONSTANTS_3RD).  The paper does not print the
// layout; this follows the block layout of ShengBTE's third-order file, extended by one atom:
//
//   <number of blocks>
//   <blank line>
//   <block number, 1-based>
//   <Cartesian position (A) of the cell of the 2nd atom: x y z>
//   <... of the 3rd atom>
//   [<... of the 4th atom>]                         (fourth order only)
//   <atom indices, 1-based: i j k [l]>
//   <alpha beta gamma [theta] value>                (27 or 81 lines, indices 1-based, eV/A^3 or eV/A^4)
//   <blank line>
//
// The first atom lies in the home cell.  Cell positions are written as n . A (A the lattice rows) and read back
// as the nearest integer n, which must reproduce the position within 1e-6 A.  Values are written with 17
// significant digits, so a write followed by a read returns every double bit for bit.
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fp_internal.cuh"

namespace {

void cell_to_cart(const double A[9], const int n[3], double out[3]) {
  for (int c = 0; c < 3; ++c) out[c] = n[0] * A[c] + n[1] * A[3 + c] + n[2] * A[6 + c];
}

// n = round(x A^-1); false if x is not a lattice vector within tol
bool cart_to_cell(const double A[9], const double x[3], int n[3]) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (std::fabs(det) < 1e-12) return false;
  // rows of inv(A): inv[r][c]; x = n A  =>  n = x inv(A)
  const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                         (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                         (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                         (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                         (A[0] * A[4] - A[1] * A[3]) / det};
  for (int a = 0; a < 3; ++a) {
    const double f = x[0] * inv[a] + x[1] * inv[3 + a] + x[2] * inv[6 + a];
    const double r = std::nearbyint(f);
    if (std::fabs(r) > 1e6) return false;
    n[a] = (int)r;
  }
  double back[3];
  cell_to_cart(A, n, back);
  for (int c = 0; c < 3; ++c)
    if (std::fabs(back[c] - x[c]) > 1e-6) return false;
  return true;
}

// One block of either order: `order` atoms (3 or 4), cells of atoms 2.. (order - 1 of them), 3^order values.
struct Block {
  int atoms[4];
  int cells[3][3];
  double fc[81];
};

int write_blocks(const char* path, const double A[9], int order, const std::vector<Block>& blocks,
                 std::string* err) {
  FILE* f = std::fopen(path, "w");
  if (!f) {
    *err = std::string("cannot open ") + path + " for writing: " + std::strerror(errno);
    return FP_EINVAL;
  }
  const int nval = order == 3 ? 27 : 81;
  std::fprintf(f, "%d\n", (int)blocks.size());
  for (size_t b = 0; b < blocks.size(); ++b) {
    const Block& k = blocks[b];
    std::fprintf(f, "\n%d\n", (int)b + 1);
    for (int r = 0; r < order - 1; ++r) {
      double x[3];
      cell_to_cart(A, k.cells[r], x);
      std::fprintf(f, "%.17g %.17g %.17g\n", x[0], x[1], x[2]);
    }
    for (int r = 0; r < order; ++r) std::fprintf(f, r ? " %d" : "%d", k.atoms[r] + 1);
    std::fprintf(f, "\n");
    for (int v = 0; v < nval; ++v) {
      int idx[4], t = v;
      for (int r = order - 1; r >= 0; --r) {
        idx[r] = t % 3;
        t /= 3;
      }
      for (int r = 0; r < order; ++r) std::fprintf(f, "%d ", idx[r] + 1);
      std::fprintf(f, "%.17g\n", k.fc[v]);
    }
  }
  const bool ok = std::ferror(f) == 0;
  if (std::fclose(f) != 0 || !ok) {
    *err = std::string("write error on ") + path;
    return FP_EINVAL;
  }
  return FP_OK;
}

int read_blocks(const char* path, const double A[9], int order, std::vector<Block>* blocks, std::string* err) {
  FILE* f = std::fopen(path, "r");
  if (!f) {
    *err = std::string("cannot open ") + path + ": " + std::strerror(errno);
    return FP_EINVAL;
  }
  auto bad = [&](const std::string& m) {
    std::fclose(f);
    *err = std::string(path) + ": " + m;
    return FP_EINVAL;
  };
  int nb = 0;
  if (std::fscanf(f, "%d", &nb) != 1 || nb < 0 || nb > 100000000) return bad("bad block count");
  const int nval = order == 3 ? 27 : 81;
  blocks->assign(nb, Block());
  for (int b = 0; b < nb; ++b) {
    Block& k = (*blocks)[b];
    int id = 0;
    if (std::fscanf(f, "%d", &id) != 1 || id != b + 1) return bad("block " + std::to_string(b + 1) + ": bad number");
    for (int r = 0; r < order - 1; ++r) {
      double x[3];
      if (std::fscanf(f, "%lf %lf %lf", &x[0], &x[1], &x[2]) != 3)
        return bad("block " + std::to_string(b + 1) + ": bad cell position");
      if (!cart_to_cell(A, x, k.cells[r]))
        return bad("block " + std::to_string(b + 1) + ": a cell position is not a lattice vector");
    }
    for (int r = 0; r < order; ++r) {
      if (std::fscanf(f, "%d", &k.atoms[r]) != 1 || k.atoms[r] < 1)
        return bad("block " + std::to_string(b + 1) + ": bad atom index");
      k.atoms[r] -= 1;
    }
    std::vector<int> seen(nval, 0);
    for (int v = 0; v < nval; ++v) {
      int idx[4];
      for (int r = 0; r < order; ++r)
        if (std::fscanf(f, "%d", &idx[r]) != 1 || idx[r] < 1 || idx[r] > 3)
          return bad("block " + std::to_string(b + 1) + ": bad Cartesian index");
      int pos = 0;
      for (int r = 0; r < order; ++r) pos = pos * 3 + (idx[r] - 1);
      double val;
      if (std::fscanf(f, "%lf", &val) != 1) return bad("block " + std::to_string(b + 1) + ": bad value");
      if (seen[pos]++) return bad("block " + std::to_string(b + 1) + ": repeated Cartesian index");
      k.fc[pos] = val;
    }
  }
  std::fclose(f);
  return FP_OK;
}

}  // namespace

extern "C" {

int fp_write_fc4(const char* path, const double lattice[9], int n, const fp_fc4* fc4) {
  std::string err;
  if (!path || !lattice || n < 0 || (n > 0 && !fc4)) return fp::fail_global(FP_EINVAL, "fp_write_fc4: bad arguments");
  std::vector<Block> blocks(n);
  for (int b = 0; b < n; ++b) {
    const fp_fc4& s = fc4[b];
    Block& k = blocks[b];
    k.atoms[0] = s.i;
    k.atoms[1] = s.j;
    k.atoms[2] = s.k;
    k.atoms[3] = s.l;
    for (int d = 0; d < 3; ++d) {
      k.cells[0][d] = s.Rj[d];
      k.cells[1][d] = s.Rk[d];
      k.cells[2][d] = s.Rl[d];
    }
    std::memcpy(k.fc, s.fc, sizeof(s.fc));
  }
  const int rc = write_blocks(path, lattice, 4, blocks, &err);
  return rc ? fp::fail_global(rc, "fp_write_fc4: " + err) : FP_OK;
}

int fp_read_fc4(const char* path, const double lattice[9], fp_fc4* out, int cap, int* n) {
  std::string err;
  if (!path || !lattice || !n || cap < 0) return fp::fail_global(FP_EINVAL, "fp_read_fc4: bad arguments");
  std::vector<Block> blocks;
  const int rc = read_blocks(path, lattice, 4, &blocks, &err);
  if (rc) return fp::fail_global(rc, "fp_read_fc4: " + err);
  *n = (int)blocks.size();
  if (!out) return FP_OK;
  if (cap < *n) return fp::fail_global(FP_EINVAL, "fp_read_fc4: the output holds fewer blocks than the file");
  for (int b = 0; b < *n; ++b) {
    const Block& k = blocks[b];
    fp_fc4& s = out[b];
    s.i = k.atoms[0];
    s.j = k.atoms[1];
    s.k = k.atoms[2];
    s.l = k.atoms[3];
    for (int d = 0; d < 3; ++d) {
      s.Rj[d] = k.cells[0][d];
      s.Rk[d] = k.cells[1][d];
      s.Rl[d] = k.cells[2][d];
    }
    std::memcpy(s.fc, k.fc, sizeof(s.fc));
  }
  return FP_OK;
}

int fp_write_fc3(const char* path, const double lattice[9], int n, const fp_fc3* fc3) {
  std::string err;
  if (!path || !lattice || n < 0 || (n > 0 && !fc3)) return fp::fail_global(FP_EINVAL, "fp_write_fc3: bad arguments");
  std::vector<Block> blocks(n);
  for (int b = 0; b < n; ++b) {
    const fp_fc3& s = fc3[b];
    Block& k = blocks[b];
    k.atoms[0] = s.i;
    k.atoms[1] = s.j;
    k.atoms[2] = s.k;
    for (int d = 0; d < 3; ++d) {
      k.cells[0][d] = s.Rj[d];
      k.cells[1][d] = s.Rk[d];
    }
    std::memcpy(k.fc, s.fc, sizeof(s.fc));
  }
  const int rc = write_blocks(path, lattice, 3, blocks, &err);
  return rc ? fp::fail_global(rc, "fp_write_fc3: " + err) : FP_OK;
}

int fp_read_fc3(const char* path, const double lattice[9], fp_fc3* out, int cap, int* n) {
  std::string err;
  if (!path || !lattice || !n || cap < 0) return fp::fail_global(FP_EINVAL, "fp_read_fc3: bad arguments");
  std::vector<Block> blocks;
  const int rc = read_blocks(path, lattice, 3, &blocks, &err);
  if (rc) return fp::fail_global(rc, "fp_read_fc3: " + err);
  *n = (int)blocks.size();
  if (!out) return FP_OK;
  if (cap < *n) return fp::fail_global(FP_EINVAL, "fp_read_fc3: the output holds fewer blocks than the file");
  for (int b = 0; b < *n; ++b) {
    const Block& k = blocks[b];
    fp_fc3& s = out[b];
    s.i = k.atoms[0];
    s.j = k.atoms[1];
    s.k = k.atoms[2];
    for (int d = 0; d < 3; ++d) {
      s.Rj[d] = k.cells[0][d];
      s.Rk[d] = k.cells[1][d];
    }
    std::memcpy(s.fc, k.fc, sizeof(s.fc));
  }
  return FP_OK;
}

}  // extern "C"
