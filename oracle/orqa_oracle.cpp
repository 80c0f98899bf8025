// ORQA oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded CPU implementation of sparse Pauli dynamics
// in the Heisenberg picture, written directly from the ORQA paper
// (arXiv 2506.13241).  Only the test suite, the smoke check and the CPU
// baseline leg of the benchmark may load this file's library; the product
// path (the CUDA library) never does, and the two share no code.
//
// Representation (Sec. II, multi-index paragraph): a Pauli string on n qubits
// is the 2n-bit multi-index I = I_1|...|I_n with the two-bit local codes
//   00 = identity, 01 = sigma_x, 10 = sigma_y, 11 = sigma_z.
// Site q (0-based) occupies bits 2q (low) and 2q+1 (high) of the integer,
// i.e. sites are counted from the right as in App. C.  The integer is held
// in four 64-bit words (little-endian word order), enough for n <= 128.
//
// The operator O = sum_I O_I sigma_I (Eq. define_O) is a std::map from the
// multi-index to a real double coefficient (App. B uses a hash map; an
// ordered map gives the same contents and a reproducible iteration order).
//
// Gate application follows Algorithm 1 (App. A), one gate (J, theta_J) at a
// time:
//   * loop over the strings; if B(I,J) is odd the local coefficient becomes
//     cos(theta) O_I and an update (I xor J, sign * sin(theta) * O_I) is
//     appended to the update list, using the value of O_I from before the
//     local update;
//   * apply the update list by insert-or-add;
//   * truncate.
// The sign of the sin term is the one of Eq. (update_rule), which indexes
// B by the destination multi-index:  O'_K = cos O_K + (-1)^((B(K,J)+1)/2)
// sin O_{K xor J}.  (Algorithm 1 prints B of the source instead; the two
// differ by a factor -1 because B(K xor J, J) = -B(K, J) mod 4.  Eq.
// (update_rule) is the one that matches U^dagger O U for U = exp(-i theta
// sigma_J / 2), which the dense-matrix tests check.)
//
// Truncation (Algorithm 1 truncate loop, absolute form): an entry is erased
// when its coefficient is exactly zero or |O_I| < delta.  The relative form
// of Eq. (truncation1), |O_I| <= eps0 * max_I |O_I|, is also provided.
//
// Rotation angles within 1e-12 of a multiple of pi/2 are treated as exact
// Clifford angles: (cos, sin) are taken from {0, +1, -1} exactly, so a
// Clifford gate maps one string to exactly one string.
//
// Expectation value in |0...0> (Eq. magnetization): <0|sigma_I|0> is 1 when
// every local code is identity or sigma_z and 0 otherwise, so
// <0|O|0> = sum of O_I over multi-indices whose local codes are all in
// {00, 11}.

#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

// The tests rebuild this file with ORACLE_MUTATION=k to plant one plausible
// mistake and check that some pin fails; the default build plants none.
//   1 source-indexed sign (Algorithm 1 as printed)   2 sin term from the updated value
//   3 no exact Clifford angles                       4 sigma_y counted as diagonal
//   5 exact zeros kept                               6 Levi-Civita orientation reversed
//   7 commuting strings rotated too                  8 relative threshold from the max before the gate
//   9 a branch overwrites an existing term           10 sin sign reversed at the Clifford angles
#ifndef ORACLE_MUTATION
#define ORACLE_MUTATION 0
#endif

namespace {

typedef std::array<uint64_t, 4> MultiIndex;

struct Operator {
    int n_qubits;
    std::map<MultiIndex, double> terms;
};

int local_code(const MultiIndex& I, int q) {
    int bit = 2 * q;
    return (int)((I[bit / 64] >> (bit % 64)) & 3u);
}

// b(I_i, J_i): 0 when either side is the identity, otherwise the sum over k
// of the Levi-Civita symbol epsilon_{I_i J_i k} with x=1, y=2, z=3.  At most
// one k contributes (the index distinct from both), so the sum is +1 for a
// cyclic pair (x,y), (y,z), (z,x), -1 for an anti-cyclic pair, 0 if equal.
int local_phase(int a, int b) {
    if (a == 0 || b == 0 || a == b) return 0;
    bool cyclic = (a == 1 && b == 2) || (a == 2 && b == 3) || (a == 3 && b == 1);
    if (ORACLE_MUTATION == 6) cyclic = !cyclic;
    return cyclic ? 1 : -1;
}

// B(I, J) = sum_i b(I_i, J_i).  Sites where J is the identity contribute 0.
int phase_exponent(const MultiIndex& I, const MultiIndex& J, int n) {
    int B = 0;
    for (int q = 0; q < n; ++q) {
        int j = local_code(J, q);
        if (j == 0) continue;
        B += local_phase(local_code(I, q), j);
    }
    return B;
}

MultiIndex xor_index(const MultiIndex& a, const MultiIndex& b) {
    MultiIndex r;
    for (int w = 0; w < 4; ++w) r[w] = a[w] ^ b[w];
    return r;
}

// B odd <=> sigma_I and sigma_J anticommute.
bool is_odd(int B) { return (B % 2) != 0; }

// (-1)^((B+1)/2) for odd B (B may be negative): +1 if B = 3 mod 4,
// -1 if B = 1 mod 4.
double update_sign(int B) {
    int m = ((B % 4) + 4) % 4;
    return (m == 3) ? 1.0 : -1.0;
}

// cos(theta), sin(theta) with exact values at multiples of pi/2.
void rotation_cos_sin(double theta, double* c, double* s) {
    const double half_pi = 1.57079632679489661923;
    double k = std::nearbyint(theta / half_pi);
    if (ORACLE_MUTATION != 3 && std::fabs(theta - k * half_pi) <= 1e-12) {
        long long m = ((long long)k % 4 + 4) % 4;
        static const double cs[4][2] = {{1.0, 0.0}, {0.0, 1.0}, {-1.0, 0.0}, {0.0, -1.0}};
        *c = cs[m][0];
        *s = (ORACLE_MUTATION == 10) ? -cs[m][1] : cs[m][1];
        return;
    }
    *c = std::cos(theta);
    *s = std::sin(theta);
}

void truncate_abs(Operator* op, double delta) {
    for (auto it = op->terms.begin(); it != op->terms.end();) {
        double v = it->second;
        bool zero = (ORACLE_MUTATION == 5) ? false : (v == 0.0);
        if (zero || std::fabs(v) < delta)
            it = op->terms.erase(it);
        else
            ++it;
    }
}

double max_abs(const Operator* op) {
    double m = 0.0;
    for (const auto& kv : op->terms) m = std::fmax(m, std::fabs(kv.second));
    return m;
}

// Relative truncation of Eq. (truncation1): drops c == 0 and |c| <= eps0 * m,
// m = max|c| over the operator after the gate's updates.
void truncate_rel(Operator* op, double eps0, double m) {
    double thr = eps0 * m;
    for (auto it = op->terms.begin(); it != op->terms.end();) {
        double v = it->second;
        if (v == 0.0 || std::fabs(v) <= thr)
            it = op->terms.erase(it);
        else
            ++it;
    }
}

// One gate of Algorithm 1 without the truncation loop.
void rotate(Operator* op, const MultiIndex& J, double theta) {
    double co, si;
    rotation_cos_sin(theta, &co, &si);
    std::vector<std::pair<MultiIndex, double>> updates;
    for (auto& kv : op->terms) {
        int B = phase_exponent(kv.first, J, op->n_qubits);
        if (ORACLE_MUTATION != 7 && !is_odd(B)) continue;
        double old = kv.second;
        kv.second = co * old;
        MultiIndex dest = xor_index(kv.first, J);
        int B_dest = phase_exponent(dest, J, op->n_qubits);
        if (ORACLE_MUTATION == 1) B_dest = B;          // source-indexed sign
        if (ORACLE_MUTATION == 2) old = kv.second;     // post-update value
        updates.push_back(std::make_pair(dest, update_sign(B_dest) * (si * old)));
    }
    for (const auto& u : updates) {
        auto it = op->terms.find(u.first);
        if (it == op->terms.end())
            op->terms.insert(u);
        else
            it->second = (ORACLE_MUTATION == 9) ? u.second : it->second + u.second;
    }
}

}  // namespace

extern "C" {

void* oracle_new(int n_qubits) {
    if (n_qubits < 1 || n_qubits > 128) return nullptr;
    Operator* op = new Operator();
    op->n_qubits = n_qubits;
    return op;
}

void oracle_free(void* h) { delete static_cast<Operator*>(h); }

// Insert-or-add one term (key: 4 words of the multi-index).
void oracle_add_term(void* h, const uint64_t* key, double c) {
    Operator* op = static_cast<Operator*>(h);
    MultiIndex I = {key[0], key[1], key[2], key[3]};
    auto it = op->terms.find(I);
    if (it == op->terms.end())
        op->terms.insert(std::make_pair(I, c));
    else
        it->second = it->second + c;
}

int64_t oracle_size(void* h) { return (int64_t)static_cast<Operator*>(h)->terms.size(); }

// Gate exp(-i theta/2 sigma_J), then truncation |c| < delta or c == 0.
void oracle_apply_gate(void* h, const uint64_t* J_words, double theta, double delta) {
    Operator* op = static_cast<Operator*>(h);
    MultiIndex J = {J_words[0], J_words[1], J_words[2], J_words[3]};
    rotate(op, J, theta);
    truncate_abs(op, delta);
}

// Same gate, then the relative truncation of Eq. (truncation1).
void oracle_apply_gate_rel(void* h, const uint64_t* J_words, double theta, double eps0) {
    Operator* op = static_cast<Operator*>(h);
    MultiIndex J = {J_words[0], J_words[1], J_words[2], J_words[3]};
    const double before = (ORACLE_MUTATION == 8) ? max_abs(op) : 0.0;
    rotate(op, J, theta);
    truncate_rel(op, eps0, ORACLE_MUTATION == 8 ? before : max_abs(op));
}

// Gate without any truncation step (exact zeros are kept).
void oracle_rotate_only(void* h, const uint64_t* J_words, double theta) {
    Operator* op = static_cast<Operator*>(h);
    MultiIndex J = {J_words[0], J_words[1], J_words[2], J_words[3]};
    rotate(op, J, theta);
}

void oracle_truncate(void* h, double delta) { truncate_abs(static_cast<Operator*>(h), delta); }

double oracle_max_abs(void* h) { return max_abs(static_cast<Operator*>(h)); }

// <0|O|0>: sum over strings with every local code in {identity, sigma_z},
// added in key order.
double oracle_expect_zero(void* h) {
    Operator* op = static_cast<Operator*>(h);
    double acc = 0.0;
    for (const auto& kv : op->terms) {
        bool diagonal = true;
        for (int q = 0; q < op->n_qubits && diagonal; ++q) {
            int a = local_code(kv.first, q);
            if (a == 1 || (ORACLE_MUTATION != 4 && a == 2)) diagonal = false;
        }
        if (diagonal) acc += kv.second;
    }
    return acc;
}

// Sum of squared coefficients (the Hilbert-Schmidt norm^2 / 2^n).
double oracle_norm2(void* h) {
    double acc = 0.0;
    for (const auto& kv : static_cast<Operator*>(h)->terms) acc += kv.second * kv.second;
    return acc;
}

// Copies up to cap terms in key order; returns the number of terms held.
int64_t oracle_export(void* h, int64_t cap, uint64_t* keys, double* coef) {
    Operator* op = static_cast<Operator*>(h);
    int64_t i = 0;
    for (const auto& kv : op->terms) {
        if (i >= cap) break;
        for (int w = 0; w < 4; ++w) keys[4 * i + w] = kv.first[w];
        coef[i] = kv.second;
        ++i;
    }
    return (int64_t)op->terms.size();
}

// Exposed for the tests of the phase rule: B(I, J).
int oracle_phase_exponent(const uint64_t* I_words, const uint64_t* J_words, int n_qubits) {
    MultiIndex I = {I_words[0], I_words[1], I_words[2], I_words[3]};
    MultiIndex J = {J_words[0], J_words[1], J_words[2], J_words[3]};
    return phase_exponent(I, J, n_qubits);
}

void oracle_rotation_cos_sin(double theta, double* c, double* s) { rotation_cos_sin(theta, c, s); }

}  // extern "C"
