// Host-side scene preprocessing: turns ipc_scene_desc arrays into the flat,
// env-concatenated tables the kernels read.
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ipc_b300.h"

namespace ipc {

enum RowKind : uint8_t {
  ROW_FREE = 0,      // free gel vertex
  ROW_PINNED = 1,    // gel vertex held at its position (eliminated)
  ROW_ATTACHED = 2,  // gel vertex driven by a body target (augmented Lagrangian)
  ROW_BODY = 3,      // sub-row of a free affine body
  ROW_BODY_DRIVEN = 4,
  ROW_PAD = 5
};

constexpr int MAX_OBJECTS_PER_ENV = 64;

struct EnvInfo {
  int n_verts = 0, n_tets = 0, n_bodies = 0, n_pads = 0;
  int row_begin = 0, n_rows = 0;       // padded rows (multiple of 128)
  int gel_rows = 0;                    // rows before the body block (multiple of 32)
  int tet_begin = 0;
  int cv_begin = 0, n_cv = 0;
  int tri_begin = 0, n_tri = 0, edge_begin = 0, n_edge = 0;
  int obj_begin = 0, n_obj = 0;
  int body_begin = 0;
  int chunk_begin = 0, n_chunks = 0;
  int coated_begin = 0, n_coated = 0;
  int pair_cap = 0;
  long long pair_begin = 0;
  std::vector<int> perm;      // internal row (local) -> user vertex id
  std::vector<int> inv_perm;  // user vertex id -> internal row (local)
  std::vector<double> body_com;   // [n_bodies][3]
  std::vector<int> body_nv;
};

struct EnvLocal;  // one env's own tables (scene.cpp)

// Flat host tables for all envs (device copies mirror these names).
struct Pack {
  std::vector<std::shared_ptr<EnvLocal>> locals;  // per env (identical consecutive scenes share one)
  int n_envs = 0;
  int n_rows = 0, n_tets = 0, n_cv = 0, n_tri = 0, n_edge = 0, n_obj = 0, n_bodies = 0;
  int n_chunks = 0, n_coated = 0;
  long long n_sell_blocks = 0;  // sum over chunks of slots * 32
  long long n_pairs_cap = 0;
  std::vector<EnvInfo> env;

  // per env
  std::vector<int> env_row_off, env_tet_off, env_cv_off, env_tri_off, env_edge_off, env_obj_off,
      env_body_off, env_chunk_off, env_coated_off;
  std::vector<long long> env_pair_off;
  std::vector<int> env_pair_cap;
  std::vector<double> env_mu, env_lam;
  std::vector<int> cta_env;  // row CTA (128 rows) -> env

  // per row
  std::vector<double> row_mass;     // gel lumped mass (0 for body / pad rows)
  std::vector<uint8_t> row_kind;
  std::vector<int> row_body;        // body sub-rows and attached rows: global body index, else -1
  std::vector<double> row_xbar;     // attached rows: [3] offset from the body's rest com
  std::vector<double> rest_x;       // initial state in row space: gel x, body y rows
  // gradient gather (gel rows): tet*4 + a, CSR over rows
  std::vector<int> vt_ptr, vt_src;

  // per tet
  std::vector<int> tets;            // [n][4] global rows
  std::vector<double> Dm_inv;       // [n][9]
  std::vector<double> tet_vol;

  // SELL-32
  std::vector<int> chunk_slots;     // per chunk
  std::vector<long long> chunk_ptr; // per chunk: offset in blocks (slot-major, 32 lanes each)
  std::vector<int> sell_col;        // [n_sell_blocks] global column row
  std::vector<int> asm_ptr;         // [n_sell_blocks + 1]
  std::vector<int> asm_src;         // tet*16 + a*4 + b

  // bodies
  std::vector<int> body_row, body_env, body_cv_begin, body_nv;
  std::vector<double> body_mass, body_S, body_vol, body_kappa;
  std::vector<uint8_t> body_driven;

  // contact vertices
  std::vector<int> cv_row, cv_body, cv_obj, cv_uid;
  std::vector<double> cv_xbar, cv_area;
  std::vector<uint8_t> cv_fixed;
  std::vector<int> tri, tri_obj;              // [n][3] global cv
  std::vector<int> edge, edge_obj;            // [n][2] global cv
  std::vector<double> edge_area, edge_len2;
  // objects
  std::vector<int> obj_env, obj_local, obj_cv_begin, obj_cv_end, obj_tri_begin, obj_tri_end,
      obj_edge_begin, obj_edge_end, obj_size;
  std::vector<unsigned long long> obj_exclude;  // bit j: never pair with env-local object j;
                                                // own bit clear: self-contact
  // coated surface rows (read_gel_surface)
  std::vector<int> coated_row;
  // broad-phase hierarchy per primitive kind k (0 contact points, 1
  // triangles, 2 edges): bv_perm[k] holds each object's primitives (global
  // ids, in the object's own range) in Morton order of their rest
  // centroids; cluster j of object o covers positions 32 j .. 32 j + 31 of
  // that order, supercluster j' its clusters 32 j' .. 32 j' + 31.
  std::vector<int> bv_perm[3];
  std::vector<int> bv_cl_obj[3], bv_sc_obj[3];      // object of each cluster / supercluster
  std::vector<int> obj_cl_begin[3], obj_sc_begin[3];  // first cluster / supercluster of each object
};

// Validates and preprocesses; returns false with a message on bad input.
bool build_pack(const ipc_scene_desc* scenes, int n_envs, const ipc_params& prm, Pack& pk,
                std::string& err);

// One env's own build (EnvLocal), for replacing an env in place:
// same_topology tells whether a new scene fits the env's segments, and
// patch_env_values writes its value tables into the flat host tables.
bool build_env_local(const ipc_scene_desc& s, int e, const ipc_params& prm, std::shared_ptr<EnvLocal>& out,
                     std::string& err);
bool same_topology(const EnvLocal& a, const EnvLocal& b);
void patch_env_values(Pack& pk, int e, const EnvLocal& L);

}  // namespace ipc
